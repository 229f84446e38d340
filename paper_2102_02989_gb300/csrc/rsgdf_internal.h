// Internal declarations of the RSGDF library (host planner <-> CUDA kernels).
#pragma once
#include <cstdint>
#include <string>
#include <functional>
#include <vector>

#include "../../include/rsgdf.h"

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace rsgdf {

constexpr int LMAX = RSGDF_LMAX;
constexpr int LTOT_MAX = 3 * LMAX;              // highest total angular momentum of a triple
constexpr int NC_MAX = (LMAX + 1) * (LMAX + 2) / 2;
constexpr int NBIN_MAX = 128;                    // largest k-mesh (BvK cells) supported
constexpr double SCREEN_DR = 1.0;                // window width of the R12 cutoffs (Bohr)
constexpr double SCREEN_EPS_PRIME = 1e-4;        // truncation of S_h (Supplementary Material)

// Boys table, one block per class L = 0..LTOT_MAX: rows i = 0..BOYS_NT-1 at
// T_i = i * BOYS_H.  Row layout: [0] T_i; classes L <= 1: Taylor blocks
// F_{m+k}(T_i)/k!, k < BOYS_TAYLOR, for m = 0..L; classes L >= 2: the block
// of m = L, then e^{-T_i}/k! (the device recurs downward from F_L).
constexpr double BOYS_H = 0.1;
constexpr int BOYS_NT = 1001;                   // T_i up to 100
constexpr double BOYS_TMAX = 99.9;              // table below, power law above (e^{-T} < 1e-43)
constexpr int BOYS_TAYLOR = 8;
constexpr int BOYS_NF = LTOT_MAX + BOYS_TAYLOR + 1;   // orders the generator evaluates
constexpr int BOYS_W = 18;                      // doubles per row (1 + 2 blocks, padded to 16 bytes)
constexpr int ENT_HDR = 8;                      // header doubles of a pair entry

__host__ __device__ constexpr inline int ncart(int l) { return (l + 1) * (l + 2) / 2; }
__host__ __device__ constexpr inline int ntuv(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }

struct Lattice {
    double a[3][3];
    double b[3][3];
    double vol;
    int nk[3];
    int Nk;
    double r_round;   // max distance of a point to the lattice point of its rounded coordinates
    int nnf;          // lattice points within 3 Omega^{1/3}
};

struct HBasis {
    int nshell = 0;
    std::vector<int> l, nprim, poff, foff;
    std::vector<double> center, exps, cn;  // cn: normalised contraction coefficients
    int nfunc = 0;
};

// One screened SR triple (aux shell P, "AO" shells mu, nu).
struct SRTriple {
    int P, mu, nu, pair;
    int L;
    int nwin, win_off;
    int nd;           // leading entries of the pair's sorted d list with R12 <= R12_max
    int nsph;         // leading entries of the sphere list with |l| <= Rc_cut + r_round
    double Rc_cut, amu, anu;
    long long item_off;
    double log10A, beta, eta1, eta2, aP;   // the s-type estimate of the Supplementary Material
};

struct SRPlan {
    std::vector<SRTriple> tri;           // sorted by L
    std::vector<double> win;             // R12 cutoffs per window
    std::vector<int> pair_doff;          // [npair+1]
    std::vector<int> dlist;              // int3 per d, sorted by R12 per pair
    std::vector<int> sph;                // int3 per lattice vector sorted by length
    std::vector<double> sph_len;
    std::vector<int> class_tri_begin;    // per L: first triple index, size LTOT_MAX+2
    long long n_items = 0;
};

// Host planner entry points (planner.cpp)
int make_lattice(const rsgdf_cell *cell, Lattice &L, std::string &err);
int load_basis(const rsgdf_basis *b, HBasis &h, std::string &err, bool allow_empty = false);
// basis made of the aux shells followed by one unit s function (exponent 0)
void unit_partner_basis(const HBasis &aux, HBasis &out);
int derive_params(const Lattice &L, const rsgdf_opts *o, double &omega, int gmesh[3], std::string &err);
// j3c SR plan for aux shells [s0, s1)
// keep(P, mu, nu), when given, restricts the plan to the triples it accepts
void plan_sr3c(const Lattice &L, const HBasis &ao, const HBasis &aux, int s0, int s1, double omega,
               double eps, SRPlan &plan, const std::function<bool(int, int, int)> &keep = {});
// compact/diffuse split of a basis at alpha_cut (primitives with exponent > alpha_cut are compact)
struct SplitBasis {
    std::vector<int> l, nprim, prim_off, parent, kind;   // kind 0 compact, 1 diffuse
    std::vector<double> center, exps, coeffs, weight;    // weight: coefficient of the sub-shell in its parent
    rsgdf_basis view() const
    {
        rsgdf_basis b;
        b.nshell = (int)l.size();
        b.l = l.data();
        b.nprim = nprim.data();
        b.prim_off = prim_off.data();
        b.center = center.data();
        b.exps = exps.data();
        b.coeffs = coeffs.data();
        return b;
    }
};
int split_basis(const rsgdf_basis *b, double acut, SplitBasis &out, std::string &err);
// j2c SR plan: "AO" basis = aux + unit partner, pairs (Q, unit)
void plan_sr2c(const Lattice &L, const HBasis &aux, const HBasis &auxu, double omega, double eps,
               SRPlan &plan);
void boys_table(std::vector<double> &tab);  // [LTOT_MAX+1][BOYS_NT][BOYS_W]
void single_E_host(int lc, double g, double *E);   // [(LMAX+1)^2]
// AFT pair screening: list of d per AO shell pair with some primitive pair above eps
void plan_pairs(const Lattice &L, const HBasis &ao, double eps, std::vector<int> &pair_doff,
                std::vector<int> &dlist);
long long sr_term_flops(int L);   // algorithmic FP64 flops of one SR term of total angular momentum L

}  // namespace rsgdf
