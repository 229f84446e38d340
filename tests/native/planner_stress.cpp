// Test driver for the host planner (tests/test_planner_pool.py): plans the SR
// sums of j3c and j2c from two host threads at once, many times, and counts
// the plans that differ from the first (a serial one).  The planner's parallel
// loops share one pool of worker threads; every plan must come out the same.
#include <cstdio>
#include <thread>

#include "rsgdf_internal.h"

using namespace rsgdf;

static double plan_digest(const Lattice &L, const HBasis &ao, const HBasis &ax, const HBasis &axu, double omega,
                          double eps)
{
    SRPlan p3, p2;
    plan_sr3c(L, ao, ax, 0, ax.nshell, omega, eps, p3);
    plan_sr2c(L, ax, axu, omega, eps, p2);
    double h = 0.0;
    for (const SRTriple &t : p3.tri) h = h * 1.000001 + t.Rc_cut + 3.0 * t.nd + 7.0 * t.nwin + t.amu;
    for (double w : p3.win) h = h * 1.0000001 + w;
    for (const SRTriple &t : p2.tri) h = h * 1.000001 + t.Rc_cut;
    return h;
}

extern "C" int planner_stress(const rsgdf_cell *cell, const rsgdf_basis *ao_in, const rsgdf_basis *aux_in,
                              double omega, double eps, int reps)
{
    std::string err;
    Lattice L;
    HBasis ao, ax, axu;
    if (make_lattice(cell, L, err) || load_basis(ao_in, ao, err) || load_basis(aux_in, ax, err)) return -1;
    unit_partner_basis(ax, axu);
    const double ref = plan_digest(L, ao, ax, axu, omega, eps);
    int bad = 0;
    for (int r = 0; r < reps; r++) {
        double h1 = 0.0, h2 = 0.0;
        std::thread t([&] { h1 = plan_digest(L, ao, ax, axu, omega, eps); });
        h2 = plan_digest(L, ao, ax, axu, omega, eps);
        t.join();
        bad += (h1 != ref) + (h2 != ref);
    }
    return bad;
}
