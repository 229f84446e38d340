// Host planner of the RSGDF library: lattice and k-mesh, basis normalisation,
// the Supplementary Material's screening of the SR double lattice sum, work
// lists for the kernels, the Boys-function table and the omega / G-box rule.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <cstring>
#include <numeric>

#include "rsgdf_internal.h"

namespace rsgdf {

static const double PI = 3.141592653589793238462643383279502884;

int make_lattice(const rsgdf_cell *cell, Lattice &L, std::string &err)
{
    if (!cell) { err = "cell is NULL"; return RSGDF_EINVAL; }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) L.a[i][j] = cell->a[3 * i + j];
    const double(*a)[3] = L.a;
    double c[3][3];  // c[i] = a_{i+1} x a_{i+2}
    for (int i = 0; i < 3; i++) {
        const double *u = a[(i + 1) % 3], *v = a[(i + 2) % 3];
        c[i][0] = u[1] * v[2] - u[2] * v[1];
        c[i][1] = u[2] * v[0] - u[0] * v[2];
        c[i][2] = u[0] * v[1] - u[1] * v[0];
    }
    double det = a[0][0] * c[0][0] + a[0][1] * c[0][1] + a[0][2] * c[0][2];
    if (!(std::fabs(det) > 1e-8)) { err = "lattice vectors are degenerate"; return RSGDF_EINVAL; }
    L.vol = std::fabs(det);
    for (int i = 0; i < 3; i++)
        for (int x = 0; x < 3; x++) L.b[i][x] = 2.0 * PI * c[i][x] / det;
    L.Nk = 1;
    for (int i = 0; i < 3; i++) {
        if (cell->kmesh[i] < 1) { err = "kmesh entries must be >= 1"; return RSGDF_EINVAL; }
        L.nk[i] = cell->kmesh[i];
        L.Nk *= cell->kmesh[i];
    }
    if (L.Nk > NBIN_MAX) { err = "k-mesh larger than 128 points is not supported"; return RSGDF_ENOTIMPL; }
    // rounding the fractional coordinates leaves |f_i| <= 1/2: the farthest
    // point is a corner of that cube
    L.r_round = 0.0;
    for (int s = 0; s < 8; s++) {
        double v[3] = {0, 0, 0};
        for (int i = 0; i < 3; i++) {
            double f = (s >> i & 1) ? 0.5 : -0.5;
            for (int x = 0; x < 3; x++) v[x] += f * a[i][x];
        }
        L.r_round = std::max(L.r_round, std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
    }
    // near-field cells: lattice points within 3 Omega^{1/3}
    double rad = 3.0 * std::cbrt(L.vol);
    int n[3];
    for (int i = 0; i < 3; i++) {
        double bl = std::sqrt(L.b[i][0] * L.b[i][0] + L.b[i][1] * L.b[i][1] + L.b[i][2] * L.b[i][2]);
        n[i] = (int)std::ceil(rad * bl / (2 * PI)) + 1;
    }
    L.nnf = 0;
    for (int i = -n[0]; i <= n[0]; i++)
        for (int j = -n[1]; j <= n[1]; j++)
            for (int k = -n[2]; k <= n[2]; k++) {
                double v[3];
                for (int x = 0; x < 3; x++) v[x] = i * a[0][x] + j * a[1][x] + k * a[2][x];
                if (std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) <= rad) L.nnf++;
            }
    return RSGDF_OK;
}

static double dfact_odd(int n)
{
    double r = 1.0;
    while (n > 1) { r *= n; n -= 2; }
    return r;
}

// radial norm of the x^l component of a primitive
static double xl_norm(double a, int l)
{
    return std::sqrt(std::pow(2.0 * a / PI, 1.5) * std::pow(4.0 * a, l) / dfact_odd(2 * l - 1));
}

int load_basis(const rsgdf_basis *b, HBasis &h, std::string &err, bool allow_empty)
{
    if (!b) { err = "basis is NULL"; return RSGDF_EINVAL; }
    if (b->nshell < (allow_empty ? 0 : 1)) { err = "basis has no shells"; return RSGDF_EINVAL; }
    if (b->nshell > 0 && (!b->l || !b->nprim || !b->prim_off || !b->center || !b->exps || !b->coeffs)) {
        err = "basis array pointer is NULL";
        return RSGDF_EINVAL;
    }
    h.nshell = b->nshell;
    h.l.assign(b->l, b->l + b->nshell);
    h.nprim.assign(b->nprim, b->nprim + b->nshell);
    h.poff.clear();
    h.foff.clear();
    h.center.assign(b->center, b->center + 3 * b->nshell);
    h.exps.clear();
    h.cn.clear();
    int f = 0;
    for (int s = 0; s < b->nshell; s++) {
        int l = b->l[s], np = b->nprim[s], o = b->prim_off[s];
        if (l < 0 || l > LMAX) { err = "shell angular momentum outside 0..3"; return RSGDF_EINVAL; }
        if (np < 1 || o < 0) { err = "shell needs at least one primitive"; return RSGDF_EINVAL; }
        h.poff.push_back((int)h.exps.size());
        h.foff.push_back(f);
        f += ncart(l);
        double self = 0.0;
        std::vector<double> c(np);
        for (int i = 0; i < np; i++) {
            double e = b->exps[o + i];
            if (!(e > 0.0) || !std::isfinite(e)) { err = "exponents must be positive"; return RSGDF_EINVAL; }
            c[i] = b->coeffs[o + i] * xl_norm(e, l);
        }
        for (int i = 0; i < np; i++)
            for (int j = 0; j < np; j++) {
                double p = b->exps[o + i] + b->exps[o + j];
                // int x^{2l} e^{-p x^2} dx * (int e^{-p y^2} dy)^2
                self += c[i] * c[j] * dfact_odd(2 * l - 1) / std::pow(2.0 * p, l) * std::pow(PI / p, 1.5);
            }
        if (!(self > 0.0)) { err = "contracted shell has zero norm"; return RSGDF_EINVAL; }
        double nc = 1.0 / std::sqrt(self);
        for (int i = 0; i < np; i++) {
            h.exps.push_back(b->exps[o + i]);
            h.cn.push_back(nc * c[i]);
        }
    }
    h.nfunc = f;
    return RSGDF_OK;
}

void unit_partner_basis(const HBasis &aux, HBasis &out)
{
    out = aux;
    out.nshell = aux.nshell + 1;
    out.l.push_back(0);
    out.nprim.push_back(1);
    out.poff.push_back((int)aux.exps.size());
    out.foff.push_back(aux.nfunc);
    out.center.push_back(0.0);
    out.center.push_back(0.0);
    out.center.push_back(0.0);
    out.exps.push_back(0.0);   // the constant function 1
    out.cn.push_back(1.0);
    out.nfunc = aux.nfunc + 1;
}

// The G box must contain the sphere |G + k12| <= G_cut for every k12 folded
// to [-1/2, 1/2) in fractional coordinates; G_cut = 2 omega sqrt(-ln eps_lr)
// is where e^{-q^2/4 omega^2} falls below eps_lr.
int derive_params(const Lattice &L, const rsgdf_opts *o, double &omega, int gmesh[3], std::string &err)
{
    if (!(o->eps_lr > 0.0 && o->eps_lr < 1.0)) { err = "eps_lr must be in (0, 1)"; return RSGDF_EINVAL; }
    double lg = std::sqrt(-std::log(o->eps_lr));
    bool have_g = o->gmesh[0] > 0 && o->gmesh[1] > 0 && o->gmesh[2] > 0;
    if (o->omega > 0.0) {
        omega = o->omega;
        if (have_g) {
            for (int i = 0; i < 3; i++) {
                if (o->gmesh[i] % 2 == 0) { err = "gmesh entries must be odd"; return RSGDF_EINVAL; }
                gmesh[i] = o->gmesh[i];
            }
        } else {
            double gc = 2.0 * omega * lg;
            for (int i = 0; i < 3; i++) {
                double al = std::sqrt(L.a[i][0] * L.a[i][0] + L.a[i][1] * L.a[i][1] + L.a[i][2] * L.a[i][2]);
                double sh = L.nk[i] > 1 ? 0.5 : 0.0;
                gmesh[i] = 2 * (int)std::ceil(gc * al / (2 * PI) + sh) + 1;
            }
        }
    } else {
        if (!have_g) { err = "either omega > 0 or a G mesh must be given"; return RSGDF_EINVAL; }
        double cov = 1e300;
        for (int i = 0; i < 3; i++) {
            if (o->gmesh[i] % 2 == 0) { err = "gmesh entries must be odd"; return RSGDF_EINVAL; }
            gmesh[i] = o->gmesh[i];
            double al = std::sqrt(L.a[i][0] * L.a[i][0] + L.a[i][1] * L.a[i][1] + L.a[i][2] * L.a[i][2]);
            double half = (o->gmesh[i] - 1) / 2.0 - (L.nk[i] > 1 ? 0.5 : 0.0);
            cov = std::min(cov, 2 * PI * half / al);
        }
        if (!(cov > 0.0)) { err = "G mesh too small for this k-mesh"; return RSGDF_EINVAL; }
        omega = cov / (2.0 * lg);
    }
    if ((long long)gmesh[0] * gmesh[1] * gmesh[2] > 4000000LL) { err = "G box too large"; return RSGDF_EINVAL; }
    return RSGDF_OK;
}

// ---------------------------------------------------------------------------
// Screening of the SR double lattice sum (Supplementary Material).
// ---------------------------------------------------------------------------

namespace {

// Worker threads kept for the life of the process: a parallel loop costs a
// wake-up instead of creating and joining threads (which took longer than
// the planning loops themselves).  One loop runs at a time; a loop started
// while another is running runs serially in its caller.  Each loop has its
// own index counter, published while its caller hands out work and withdrawn
// (under the lock) before the caller waits for the workers that joined: a
// worker that wakes late finds no loop and cannot take indices of the next.
class WorkerPool {
public:
    explicit WorkerPool(int nt)
    {
        for (int t = 0; t < nt; t++) th_.emplace_back([this] { work(); });
    }
    ~WorkerPool()
    {
        {
            std::lock_guard<std::mutex> lk(m_);
            quit_ = true;
        }
        cv_.notify_all();
        for (auto &t : th_) t.join();
    }
    void run(int n, const std::function<void(int)> &f)
    {
        std::unique_lock<std::mutex> own(busy_, std::try_to_lock);
        if (!own.owns_lock() || th_.empty()) {
            for (int i = 0; i < n; i++) f(i);
            return;
        }
        Loop loop{&f, n};
        {
            std::lock_guard<std::mutex> lk(m_);
            loop_ = &loop;
            gen_++;
        }
        cv_.notify_all();
        loop.drain();
        std::unique_lock<std::mutex> lk(m_);
        loop_ = nullptr;
        done_.wait(lk, [&] { return active_ == 0; });
    }

private:
    struct Loop {
        const std::function<void(int)> *f;
        int n;
        std::atomic<int> next{0};
        void drain()
        {
            for (int i; (i = next.fetch_add(1)) < n;) (*f)(i);
        }
    };
    void work()
    {
        long seen = 0;
        for (;;) {
            std::unique_lock<std::mutex> lk(m_);
            cv_.wait(lk, [&] { return quit_ || (loop_ && gen_ != seen); });
            if (quit_) return;
            Loop *loop = loop_;
            seen = gen_;
            active_++;
            lk.unlock();
            loop->drain();
            lk.lock();
            if (--active_ == 0) done_.notify_all();
        }
    }
    std::vector<std::thread> th_;
    std::mutex m_, busy_;
    std::condition_variable cv_, done_;
    Loop *loop_ = nullptr;
    long gen_ = 0;
    int active_ = 0;
    bool quit_ = false;
};

WorkerPool &worker_pool()
{
    static WorkerPool pool(std::max(0, std::min((int)std::thread::hardware_concurrency(), 32) - 1));
    return pool;
}

// dynamic partition of [0, n) over the pool and the calling thread
template <class F>
void parallel_for(int n, F f)
{
    if (n < 64) {
        for (int i = 0; i < n; i++) f(i);
        return;
    }
    const std::function<void(int)> g(f);
    worker_pool().run(n, g);
}

struct Vec3 { double x, y, z; };
inline Vec3 lat(const Lattice &L, int i, int j, int k)
{
    return {i * L.a[0][0] + j * L.a[1][0] + k * L.a[2][0], i * L.a[0][1] + j * L.a[1][1] + k * L.a[2][1],
            i * L.a[0][2] + j * L.a[1][2] + k * L.a[2][2]};
}
inline double len(Vec3 v) { return std::sqrt(v.x * v.x + v.y * v.y + v.z * v.z); }

// integer box covering the ball of radius r around point c
void ball_box(const Lattice &L, Vec3 c, double r, int lo[3], int hi[3])
{
    for (int i = 0; i < 3; i++) {
        double bl = std::sqrt(L.b[i][0] * L.b[i][0] + L.b[i][1] * L.b[i][1] + L.b[i][2] * L.b[i][2]);
        double f = (c.x * L.b[i][0] + c.y * L.b[i][1] + c.z * L.b[i][2]) / (2 * PI);
        double e = r * bl / (2 * PI);
        lo[i] = (int)std::floor(f - e) - 1;
        hi[i] = (int)std::ceil(f + e) + 1;
    }
}

int diffuse_index(const HBasis &b, int s)
{
    int o = b.poff[s], best = o;
    for (int i = 1; i < b.nprim[s]; i++)
        if (b.exps[o + i] < b.exps[best]) best = o + i;
    return best;
}

// weight of a primitive treated as a normalised 1s of the same exponent
double w1s(const HBasis &b, int s, int idx)
{
    double e = b.exps[idx];
    return std::fabs(b.cn[idx]) * std::pow(2.0 * e / PI, 0.75) / xl_norm(e, b.l[s]);
}

// Growth of a Cartesian pair of degrees (lm, ln) with separation R, and of the
// erfc tail seen by degrees lP and lpair at distance R, relative to s functions.
inline double ipow(double x, int n)
{
    double r = 1.0;
    for (int i = 0; i < n; i++) r *= x;
    return r;
}
inline double grow_r12(int lm, int ln, double am, double an, double R)
{
    double p = am + an;
    return ipow(1.0 + std::sqrt(4.0 * am) * an / p * R, lm) * ipow(1.0 + std::sqrt(4.0 * an) * am / p * R, ln);
}
inline double grow_rc(int lP, int lpair, double aP, double p, double eta2, double R)
{
    double x = 2.0 * eta2 * eta2 * R;
    return ipow(1.0 + x / std::sqrt(aP), lP) * ipow(1.0 + x / std::sqrt(p), lpair);
}

// Eq. Ncell with dR = 1 Bohr
inline double cells_in_shell(const Lattice &L, double R)
{
    double R0 = std::sqrt(L.nnf * L.vol / (8 * PI * SCREEN_DR)) - SCREEN_DR;
    if (R > R0) return 8.0 * PI / L.vol * (R + SCREEN_DR) * (R + SCREEN_DR) * SCREEN_DR;
    return (double)L.nnf;
}

// Images of the pair separation vector sorted by length (distances only).
struct PairImages { std::vector<double> r; };

void pair_images(const Lattice &L, Vec3 d0, double rmax, PairImages &out)
{
    int lo[3], hi[3];
    ball_box(L, {-d0.x, -d0.y, -d0.z}, rmax, lo, hi);
    out.r.clear();
    for (int i = lo[0]; i <= hi[0]; i++)
        for (int j = lo[1]; j <= hi[1]; j++)
            for (int k = lo[2]; k <= hi[2]; k++) {
                Vec3 v = lat(L, i, j, k);
                double r = len({v.x + d0.x, v.y + d0.y, v.z + d0.z});
                if (r <= rmax) out.r.push_back(r);
            }
    std::sort(out.r.begin(), out.r.end());
}

// bisection for the outer root of a function that is >= eps at lo and < eps
// at hi, to 1e-10 relative (the radii are compared with distances of order
// 1-100 Bohr)
template <class F>
double outer_root(F f, double lo, double hi, double eps)
{
    for (int it = 0; it < 200 && hi - lo > 1e-10 * hi; it++) {
        double mid = 0.5 * (lo + hi);
        if (f(mid) >= eps) lo = mid; else hi = mid;
    }
    return hi;
}

struct Bounds {
    double Rc_cut;
    std::vector<double> r12;  // per window
    double r12_max;
    double amu, anu;
    double log10A, beta, eta1, eta2, aP;
};

// Everything of the bounds that depends only on the AO shell pair.
struct PairPart {
    double am, an, p, beta;
    int lm, ln;
    double qp;        // sum over primitive pairs of the 1s weights / p^{3/2}
    double Sh;        // Eq. S_h (with the growth factor), never below the largest term
    double r12min;    // Eq. R12cutmin
    double xm;        // argmax of x e^{-beta x^2} grow(x), the left bracket of Eq. bound_R12_FF
    // shape(x) = x e^{-beta x^2} grow(x) at x = xm + j dx, j = 0..NSHAPE (decreasing):
    // brackets the root of every window of Eq. bound_R12_FF (c1 shape(x) = eps)
    static constexpr int NSHAPE = 256;
    double dx;
    double shape[NSHAPE + 1];
};

void pair_part(const Lattice &L, const HBasis &ao, int mu, int nu, PairPart &Q)
{
    int im = diffuse_index(ao, mu), in = diffuse_index(ao, nu);
    double am = ao.exps[im], an = ao.exps[in];
    int lm = ao.l[mu], ln = ao.l[nu];
    double p = am + an, beta = am * an / p;
    Q.am = am; Q.an = an; Q.p = p; Q.beta = beta; Q.lm = lm; Q.ln = ln;
    Q.qp = 0.0;
    for (int i = 0; i < ao.nprim[mu]; i++)
        for (int j = 0; j < ao.nprim[nu]; j++) {
            int oi = ao.poff[mu] + i, oj = ao.poff[nu] + j;
            Q.qp += w1s(ao, mu, oi) * w1s(ao, nu, oj) / std::pow(ao.exps[oi] + ao.exps[oj], 1.5);
        }
    Vec3 d0 = {ao.center[3 * nu] - ao.center[3 * mu], ao.center[3 * nu + 1] - ao.center[3 * mu + 1],
               ao.center[3 * nu + 2] - ao.center[3 * mu + 2]};
    double rprime = std::sqrt(-std::log(SCREEN_EPS_PRIME) / beta);   // h(R) = eps' radius
    PairImages img;
    pair_images(L, d0, rprime + 1e-9, img);
    auto hfun = [&](double R) { return std::exp(-beta * R * R) * grow_r12(lm, ln, am, an, R); };
    double Sh = 0.0, hbig = 0.0;
    std::vector<double> hv(img.r.size());
    for (size_t i = 0; i < img.r.size(); i++) {
        double r = img.r[i];
        hv[i] = hfun(r);
        if (std::exp(-beta * r * r) >= SCREEN_EPS_PRIME) Sh += hv[i];
        hbig = std::max(hbig, hv[i]);
    }
    if (img.r.empty()) {   // no image within the eps' radius: take the nearest one
        PairImages near;
        double rr = rprime;
        do { rr *= 2; pair_images(L, d0, rr, near); } while (near.r.empty());
        hbig = hfun(near.r[0]);
    }
    Q.Sh = std::max(Sh, hbig);
    // Eq. R12cutmin: first x on a 0.01 Bohr grid where the continuum estimate
    // is no smaller than the eps'-truncated image sum beyond x (suffix sums of
    // the sorted images)
    std::vector<double> suffix(img.r.size() + 1, 0.0);
    for (size_t i = img.r.size(); i-- > 0;)
        suffix[i] = suffix[i + 1] + ((std::exp(-beta * img.r[i] * img.r[i]) >= SCREEN_EPS_PRIME) ? hv[i] : 0.0);
    double xmax = rprime + SCREEN_DR;
    Q.r12min = xmax;
    size_t pos = 0;
    for (int ix = 0;; ix++) {
        double x = 0.01 * ix;
        if (x > xmax) break;
        while (pos < img.r.size() && img.r[pos] <= x) pos++;
        double est = 4.0 * PI / L.vol * x / (2.0 * beta) * std::exp(-beta * x * x) * grow_r12(lm, ln, am, an, x);
        if (est >= suffix[pos]) { Q.r12min = x; break; }
    }
    double x0 = 1.0 / std::sqrt(2.0 * beta);
    auto shape = [&](double x) { return x * std::exp(-beta * x * x) * grow_r12(lm, ln, am, an, x); };
    Q.xm = x0;
    double vm = shape(x0);
    double step = 0.05 / std::sqrt(beta), top = x0 + 10.0 / std::sqrt(beta);
    for (int it = 0;; it++) {
        double t = it * step;
        if (!(t < top)) break;
        double v = shape(t);
        if (v > vm) { vm = v; Q.xm = t; }
    }
    Q.dx = 10.0 / std::sqrt(beta) / PairPart::NSHAPE;
    for (int j = 0; j <= PairPart::NSHAPE; j++) Q.shape[j] = shape(Q.xm + j * Q.dx);
}

// The bounds for one (aux shell P, AO shell pair) from the pair part.
void triple_bounds(const Lattice &L, double omega, double eps, const HBasis &aux, int P, const PairPart &Q,
                   Bounds &B)
{
    int iP = diffuse_index(aux, P);
    double aP = aux.exps[iP];
    int lP = aux.l[P], lm = Q.lm, ln = Q.ln;
    double p = Q.p, beta = Q.beta, am = Q.am, an = Q.an;
    double eta1 = 1.0 / std::sqrt(1.0 / aP + 1.0 / p);
    double eta2 = 1.0 / std::sqrt(1.0 / (eta1 * eta1) + 1.0 / (omega * omega));
    // s-type prefactor pi^3 C_P C_mu C_nu / (a_P p)^{3/2}, summed over the
    // primitive combinations of the contractions (decay rates stay those of
    // the most diffuse primitives)
    double qa = 0.0;
    for (int k = 0; k < aux.nprim[P]; k++) {
        int o = aux.poff[P] + k;
        qa += w1s(aux, P, o) / std::pow(aux.exps[o], 1.5);
    }
    double A = PI * PI * PI * qa * Q.qp;
    B.amu = am;
    B.anu = an;
    B.log10A = std::log10(A);
    B.beta = beta;
    B.eta1 = eta1;
    B.eta2 = eta2;
    B.aP = aP;
    // Eq. bound_Rc
    double c0 = A * Q.Sh * 4.0 * PI / L.vol / std::sqrt(PI) / (2.0 * eta2 * eta2 * eta2);
    auto grc = [&](double R) { return c0 / R * std::exp(-eta2 * eta2 * R * R) * grow_rc(lP, lm + ln, aP, p, eta2, R); };
    double hi = 1e-6;
    while (grc(hi) >= eps && hi < 1e4) hi *= 2;
    B.Rc_cut = (hi > 1e-6) ? outer_root(grc, 1e-6, hi, eps) : hi;
    // Eq. bound_R12_FF per window, then Eq. bound_R12
    int nw = (int)std::floor(B.Rc_cut / SCREEN_DR) + 1;
    nw = std::min(nw, 512);
    B.r12.assign(nw, 0.0);
    B.r12_max = 0.0;
    for (int w = 0; w < nw; w++) {
        double R = w * SCREEN_DR;
        double fR = (R < 1e-8) ? 2.0 * (eta1 - eta2) / std::sqrt(PI) : (std::erf(eta1 * R) - std::erf(eta2 * R)) / R;
        double c1 = A * cells_in_shell(L, R) * fR * grow_rc(lP, lm + ln, aP, p, eta2, R) * 4.0 * PI / L.vol / (2.0 * beta);
        auto g = [&](double x) { return c1 * x * std::exp(-beta * x * x) * grow_r12(lm, ln, am, an, x); };
        double x = 0.0;
        if (c1 * Q.shape[0] >= eps) {
            const double target = eps / c1;
            if (Q.shape[PairPart::NSHAPE] >= target) {   // beyond the table: expand the bracket
                double a = Q.xm + PairPart::NSHAPE * Q.dx, b = 2.0 * a;
                while (g(b) >= eps && b < 1e4) { a = b; b *= 2; }
                x = outer_root(g, a, b, eps);
            } else {
                int lo = 0, hi = PairPart::NSHAPE;   // shape[lo] >= target > shape[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) / 2;
                    if (Q.shape[mid] >= target) lo = mid; else hi = mid;
                }
                // safeguarded Newton on log(c1 shape(x)) - log(eps), decreasing on the bracket
                const double k1 = std::sqrt(4.0 * am) * an / p, k2 = std::sqrt(4.0 * an) * am / p;
                const double lc = std::log(c1) - std::log(eps);
                auto h = [&](double y) {
                    return lc + std::log(y) - beta * y * y + lm * std::log1p(k1 * y) + ln * std::log1p(k2 * y);
                };
                auto dh = [&](double y) { return 1.0 / y - 2.0 * beta * y + lm * k1 / (1.0 + k1 * y) + ln * k2 / (1.0 + k2 * y); };
                double a = Q.xm + lo * Q.dx, b = Q.xm + hi * Q.dx;
                double ha = std::log(Q.shape[lo] / target), hb = std::log(Q.shape[hi] / target);
                double y = (ha - hb > 0.0) ? a + (b - a) * ha / (ha - hb) : 0.5 * (a + b);
                for (int it = 0; it < 60; it++) {
                    const double hy = h(y);
                    if (hy >= 0.0) a = y; else b = y;
                    const double d = dh(y);
                    double yn = (d < 0.0) ? y - hy / d : 0.5 * (a + b);
                    if (!(yn > a && yn < b)) yn = 0.5 * (a + b);
                    const bool done = std::fabs(yn - y) <= 1e-12 * y || b - a <= 1e-12 * b;
                    y = yn;
                    if (done) break;
                }
                x = y;
            }
        }
        B.r12[w] = std::max(x, Q.r12min);
        B.r12_max = std::max(B.r12_max, B.r12[w]);
    }
}

// two-center bound: the pair replaced by the second aux function (S_h = 1)
double pair2c_cut(const Lattice &L, double omega, double eps, const HBasis &aux, int P, int Q)
{
    int iP = diffuse_index(aux, P), iQ = diffuse_index(aux, Q);
    double aP = aux.exps[iP], aQ = aux.exps[iQ];
    double eta1 = 1.0 / std::sqrt(1.0 / aP + 1.0 / aQ);
    double eta2 = 1.0 / std::sqrt(1.0 / (eta1 * eta1) + 1.0 / (omega * omega));
    double qa = 0.0, qb = 0.0;
    for (int k = 0; k < aux.nprim[P]; k++) {
        int o = aux.poff[P] + k;
        qa += w1s(aux, P, o) / std::pow(aux.exps[o], 1.5);
    }
    for (int k = 0; k < aux.nprim[Q]; k++) {
        int o = aux.poff[Q] + k;
        qb += w1s(aux, Q, o) / std::pow(aux.exps[o], 1.5);
    }
    double c0 = PI * PI * PI * qa * qb * 4.0 * PI / L.vol / std::sqrt(PI) / (2.0 * eta2 * eta2 * eta2);
    auto g = [&](double R) { return c0 / R * std::exp(-eta2 * eta2 * R * R); };
    double hi = 1e-6;
    while (g(hi) >= eps && hi < 1e4) hi *= 2;
    return (hi > 1e-6) ? outer_root(g, 1e-6, hi, eps) : hi;
}

void sphere_list(const Lattice &L, double rmax, SRPlan &plan)
{
    int lo[3], hi[3];
    ball_box(L, {0, 0, 0}, rmax, lo, hi);
    struct E { double r; int i, j, k; };
    std::vector<E> v;
    for (int i = lo[0]; i <= hi[0]; i++)
        for (int j = lo[1]; j <= hi[1]; j++)
            for (int k = lo[2]; k <= hi[2]; k++) {
                double r = len(lat(L, i, j, k));
                if (r <= rmax) v.push_back({r, i, j, k});
            }
    std::sort(v.begin(), v.end(), [](const E &x, const E &y) {
        if (x.r != y.r) return x.r < y.r;
        if (x.i != y.i) return x.i < y.i;
        if (x.j != y.j) return x.j < y.j;
        return x.k < y.k;
    });
    plan.sph.clear();
    plan.sph_len.clear();
    for (auto &e : v) {
        plan.sph.push_back(e.i);
        plan.sph.push_back(e.j);
        plan.sph.push_back(e.k);
        plan.sph_len.push_back(e.r);
    }
}

void finish_plan(const Lattice &L, SRPlan &plan)
{
    std::stable_sort(plan.tri.begin(), plan.tri.end(), [](const SRTriple &a, const SRTriple &b) { return a.L < b.L; });
    double rmax = 0.0;
    for (auto &t : plan.tri) rmax = std::max(rmax, t.Rc_cut + L.r_round);
    sphere_list(L, rmax + 1e-9, plan);
    plan.class_tri_begin.assign(LTOT_MAX + 2, 0);
    long long off = 0;
    for (size_t i = 0; i < plan.tri.size(); i++) {
        SRTriple &t = plan.tri[i];
        t.nsph = (int)(std::upper_bound(plan.sph_len.begin(), plan.sph_len.end(), t.Rc_cut + L.r_round) -
                       plan.sph_len.begin());
        t.item_off = off;
        off += t.nd;
    }
    plan.n_items = off;
    for (int c = 0; c <= LTOT_MAX + 1; c++) {
        int n = 0;
        while (n < (int)plan.tri.size() && plan.tri[n].L < c) n++;
        plan.class_tri_begin[c] = n;
    }
}

}  // namespace

void plan_sr3c(const Lattice &L, const HBasis &ao, const HBasis &aux, int s0, int s1, double omega, double eps,
               SRPlan &plan, const std::function<bool(int, int, int)> &keep)
{
    plan = SRPlan();
    int ns = ao.nshell;
    std::vector<PairPart> pp((size_t)ns * ns);
    std::vector<Bounds> bnd((size_t)(s1 - s0) * ns * ns);
    std::vector<double> pair_rmax((size_t)ns * ns, 0.0);
    parallel_for(ns * ns, [&](int pr) { pair_part(L, ao, pr / ns, pr % ns, pp[pr]); });
    parallel_for((s1 - s0) * ns * ns, [&](int id) {
        int P = s0 + id / (ns * ns), pr = id % (ns * ns);
        triple_bounds(L, omega, eps, aux, P, pp[pr], bnd[id]);
    });
    for (int P = s0; P < s1; P++)
        for (int pr = 0; pr < ns * ns; pr++)
            if (!keep || keep(P, pr / ns, pr % ns))
                pair_rmax[pr] = std::max(pair_rmax[pr], bnd[(size_t)(P - s0) * ns * ns + pr].r12_max);
    // per AO shell pair: d vectors with R12 <= max over P, sorted by R12
    plan.pair_doff.assign(ns * ns + 1, 0);
    std::vector<std::vector<double>> pair_r12(ns * ns);
    for (int mu = 0; mu < ns; mu++)
        for (int nu = 0; nu < ns; nu++) {
            int pr = mu * ns + nu;
            Vec3 c = {ao.center[3 * mu] - ao.center[3 * nu], ao.center[3 * mu + 1] - ao.center[3 * nu + 1],
                      ao.center[3 * mu + 2] - ao.center[3 * nu + 2]};
            int lo[3], hi[3];
            ball_box(L, c, pair_rmax[pr], lo, hi);
            struct D { double r; int i, j, k; };
            std::vector<D> ds;
            for (int i = lo[0]; i <= hi[0]; i++)
                for (int j = lo[1]; j <= hi[1]; j++)
                    for (int k = lo[2]; k <= hi[2]; k++) {
                        Vec3 v = lat(L, i, j, k);
                        double r = len({v.x - c.x, v.y - c.y, v.z - c.z});
                        if (r <= pair_rmax[pr]) ds.push_back({r, i, j, k});
                    }
            std::sort(ds.begin(), ds.end(), [](const D &x, const D &y) { return x.r < y.r; });
            plan.pair_doff[pr] = (int)(plan.dlist.size() / 3);
            for (auto &d : ds) {
                plan.dlist.push_back(d.i);
                plan.dlist.push_back(d.j);
                plan.dlist.push_back(d.k);
                pair_r12[pr].push_back(d.r);
            }
        }
    plan.pair_doff[ns * ns] = (int)(plan.dlist.size() / 3);
    for (int P = s0; P < s1; P++)
        for (int mu = 0; mu < ns; mu++)
            for (int nu = 0; nu < ns; nu++) {
                if (keep && !keep(P, mu, nu)) continue;
                Bounds &B = bnd[((size_t)(P - s0) * ns + mu) * ns + nu];
                int pr = mu * ns + nu;
                SRTriple t;
                t.P = P; t.mu = mu; t.nu = nu; t.pair = pr;
                t.L = aux.l[P] + ao.l[mu] + ao.l[nu];
                t.nwin = (int)B.r12.size();
                t.win_off = (int)plan.win.size();
                plan.win.insert(plan.win.end(), B.r12.begin(), B.r12.end());
                t.nd = (int)(std::upper_bound(pair_r12[pr].begin(), pair_r12[pr].end(), B.r12_max) - pair_r12[pr].begin());
                t.Rc_cut = B.Rc_cut;
                t.amu = B.amu;
                t.anu = B.anu;
                t.nsph = 0;
                t.item_off = 0;
                t.log10A = B.log10A;
                t.beta = B.beta;
                t.eta1 = B.eta1;
                t.eta2 = B.eta2;
                t.aP = B.aP;
                if (t.nd > 0) plan.tri.push_back(t);
            }
    finish_plan(L, plan);
}

void plan_sr2c(const Lattice &L, const HBasis &aux, const HBasis &auxu, double omega, double eps, SRPlan &plan)
{
    plan = SRPlan();
    int ns = auxu.nshell;     // aux shells + the unit partner
    int unit = ns - 1;
    plan.pair_doff.assign(ns * ns + 1, 0);
    // the only "pair" used is (Q, unit) with d = 0
    for (int pr = 0; pr <= ns * ns; pr++) plan.pair_doff[pr] = 0;
    std::vector<int> one = {0, 0, 0};
    for (int Q = 0; Q < aux.nshell; Q++) {
        int pr = Q * ns + unit;
        plan.pair_doff[pr] = (int)(plan.dlist.size() / 3);
        plan.dlist.insert(plan.dlist.end(), one.begin(), one.end());
        for (int q = pr + 1; q <= ns * ns; q++) plan.pair_doff[q] = (int)(plan.dlist.size() / 3);
    }
    const int na = aux.nshell;
    std::vector<double> rc((size_t)na * na);
    parallel_for(na * na, [&](int id) { rc[id] = pair2c_cut(L, omega, eps, aux, id / na, id % na); });
    for (int P = 0; P < aux.nshell; P++)
        for (int Q = 0; Q < aux.nshell; Q++) {
            SRTriple t;
            t.P = P; t.mu = Q; t.nu = unit; t.pair = Q * ns + unit;
            t.L = aux.l[P] + aux.l[Q];
            t.nwin = 1;
            t.win_off = (int)plan.win.size();
            plan.win.push_back(1e300);
            t.nd = 1;
            t.Rc_cut = rc[(size_t)P * na + Q];
            t.amu = aux.exps[diffuse_index(aux, Q)];
            t.anu = 0.0;
            t.nsph = 0;
            t.item_off = 0;
            t.log10A = 0.0;
            t.beta = 0.0;
            t.eta1 = t.eta2 = 1.0;
            t.aP = aux.exps[diffuse_index(aux, P)];
            plan.tri.push_back(t);
        }
    finish_plan(L, plan);
}

void plan_pairs(const Lattice &L, const HBasis &ao, double eps, std::vector<int> &pair_doff, std::vector<int> &dlist)
{
    int ns = ao.nshell;
    pair_doff.assign(ns * ns + 1, 0);
    dlist.clear();
    for (int mu = 0; mu < ns; mu++)
        for (int nu = 0; nu < ns; nu++) {
            int pr = mu * ns + nu;
            pair_doff[pr] = (int)(dlist.size() / 3);
            // radius beyond which no primitive pair passes
            double rmax = 0.0;
            for (int i = 0; i < ao.nprim[mu]; i++)
                for (int j = 0; j < ao.nprim[nu]; j++) {
                    int oi = ao.poff[mu] + i, oj = ao.poff[nu] + j;
                    double a = ao.exps[oi], b = ao.exps[oj], p = a + b;
                    double c = std::fabs(ao.cn[oi] * ao.cn[oj]) * std::pow(PI / p, 1.5);
                    if (c >= eps) rmax = std::max(rmax, std::sqrt(std::log(c / eps) / (a * b / p)));
                }
            Vec3 c = {ao.center[3 * mu] - ao.center[3 * nu], ao.center[3 * mu + 1] - ao.center[3 * nu + 1],
                      ao.center[3 * mu + 2] - ao.center[3 * nu + 2]};
            int lo[3], hi[3];
            ball_box(L, c, rmax, lo, hi);
            for (int i = lo[0]; i <= hi[0]; i++)
                for (int j = lo[1]; j <= hi[1]; j++)
                    for (int k = lo[2]; k <= hi[2]; k++) {
                        Vec3 v = lat(L, i, j, k);
                        double R = len({v.x - c.x, v.y - c.y, v.z - c.z});
                        // some primitive pair has |c_i c_j| (pi/p)^{3/2} e^{-ab/p R^2} >= eps
                        // exactly when R <= rmax (the largest of their radii)
                        if (rmax > 0.0 && R <= rmax) {
                            dlist.push_back(i);
                            dlist.push_back(j);
                            dlist.push_back(k);
                        }
                    }
        }
    pair_doff[ns * ns] = (int)(dlist.size() / 3);
}

// F_m(T) = e^{-T} sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)) in long double
// (every term positive), stored per class L as Taylor blocks about T_i
// (d^k F_m/dT^k = (-1)^k F_{m+k}): row i of class L holds T_i, then
// F_{m+k}(T_i)/k! for m = 0..L (L <= 1) or for m = L followed by
// e^{-T_i}/k! (L >= 2).
void boys_table(std::vector<double> &tab)
{
    tab.assign((size_t)(LTOT_MAX + 1) * BOYS_NT * BOYS_W, 0.0);
    std::vector<long double> F(BOYS_NF);
    for (int i = 0; i < BOYS_NT; i++) {
        const long double T = (long double)i * BOYS_H;
        const long double eT = expl(-T);
        for (int m = 0; m < BOYS_NF; m++) {
            long double term = 1.0L / (2 * m + 1), sum = term;
            for (int k = 1; k < 8000; k++) {
                term *= 2.0L * T / (2 * m + 2 * k + 1);
                sum += term;
                if (term < 1e-22L * sum) break;
            }
            F[m] = eT * sum;
        }
        for (int L = 0; L <= LTOT_MAX; L++) {
            double *row = &tab[((size_t)L * BOYS_NT + i) * BOYS_W];
            row[0] = (double)T;
            long double fact = 1.0L;
            for (int k = 0; k < BOYS_TAYLOR; k++) {
                if (k > 0) fact *= k;
                if (L <= 1) {
                    for (int m = 0; m <= L; m++) row[1 + m * BOYS_TAYLOR + k] = (double)(F[m + k] / fact);
                } else {
                    row[1 + k] = (double)(F[L + k] / fact);
                    row[1 + BOYS_TAYLOR + k] = (double)(eT / fact);
                }
            }
        }
    }
}

// Hermite coefficients of the single-centre Gaussian x^c e^{-g x^2}:
// E^{c+1}_t = E^c_{t-1}/(2g) + (t+1) E^c_{t+1}
void single_E_host(int lc, double g, double *E)
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

// Algorithmic FP64 flops of one SR term (one primitive combination) with
// total angular momentum L, as the kernel evaluates it: pair-centre distance
// and T (8); two Boys evaluations, each either a 7-step Taylor series per
// order (L <= 2) or one for F_L and one for e^{-T} plus a 2-flop downward step
// per order, counting an FMA as 2; the erfc combination and its seed scaling
// (3 per order); the Hermite recursion (2 flops per first-index step, 2 more
// when the (t-1) term is present); the accumulation (1 per Hermite integral).
long long sr_term_flops(int L)
{
    long long boys = (L <= 2) ? 14LL * (L + 1) : 28LL + 4LL * L;
    long long f = 8 + 2 * boys + 3 * (L + 1);
    for (int n = 0; n < L; n++)
        for (int s = 1; s <= L - n; s++)
            for (int t = 0; t <= s; t++)
                for (int u = 0; u <= s - t; u++) {
                    int v = s - t - u;
                    int lead = t > 0 ? t : (u > 0 ? u : v);
                    f += 2 + (lead > 1 ? 2 : 0);
                }
    f += ntuv(L);
    return f;
}

}  // namespace rsgdf

namespace rsgdf {

// Compact/diffuse split (Fig. 1 of the paper): every shell becomes a compact
// sub-shell (its primitives with exponent > alpha_cut) and/or a diffuse one,
// with the parent's raw coefficients; each sub-shell is normalised on its own,
// so the parent function is sum_S (n_parent / n_S) chi_S, n the contraction
// norm factor (1/sqrt of the self-overlap of the x^l component).
static double contracted_norm(int l, const double *e, const double *c, int np)
{
    double self = 0.0;
    for (int i = 0; i < np; i++)
        for (int j = 0; j < np; j++) {
            const double p = e[i] + e[j];
            self += c[i] * xl_norm(e[i], l) * c[j] * xl_norm(e[j], l) * dfact_odd(2 * l - 1) / std::pow(2.0 * p, l) *
                    std::pow(PI / p, 1.5);
        }
    return 1.0 / std::sqrt(self);
}

int split_basis(const rsgdf_basis *b, double acut, SplitBasis &out, std::string &err)
{
    HBasis h;
    const int rc = load_basis(b, h, err);
    if (rc != RSGDF_OK) return rc;
    if (!(acut >= 0.0) || !std::isfinite(acut)) {
        err = "alpha_cut must be finite and >= 0";
        return RSGDF_EINVAL;
    }
    out = SplitBasis();
    for (int s = 0; s < b->nshell; s++) {
        const int l = b->l[s], np = b->nprim[s], o = b->prim_off[s];
        const double npar = contracted_norm(l, b->exps + o, b->coeffs + o, np);
        for (int kind = 0; kind < 2; kind++) {   // 0 compact, 1 diffuse
            std::vector<double> e, c;
            for (int i = 0; i < np; i++)
                if ((b->exps[o + i] > acut) == (kind == 0)) {
                    e.push_back(b->exps[o + i]);
                    c.push_back(b->coeffs[o + i]);
                }
            if (e.empty()) continue;
            out.l.push_back(l);
            out.nprim.push_back((int)e.size());
            out.prim_off.push_back((int)out.exps.size());
            for (int x = 0; x < 3; x++) out.center.push_back(b->center[3 * s + x]);
            out.exps.insert(out.exps.end(), e.begin(), e.end());
            out.coeffs.insert(out.coeffs.end(), c.begin(), c.end());
            out.parent.push_back(s);
            out.kind.push_back(kind);
            out.weight.push_back(npar / contracted_norm(l, e.data(), c.data(), (int)e.size()));
        }
    }
    return RSGDF_OK;
}

}  // namespace rsgdf
