// Host check of the projection's seed tables (flic::build_proj_tables_into): wherever a
// seed decides a bin without the sign tests, the point lies more than 1e-6 rad from every
// boundary and in the exact bin.  The kernel's arithmetic is emulated in fp32 with its
// worst-case seed errors: t = tan(elevation) within 2.4e-7 |t| (z * rsqrt(rho^2)), the
// azimuth seed within 1.1e-6 rad.
//   seed_table_check R C seed trials [mode]   mode 0: random elevations, 1: unsorted,
//                                              2: narrow field, 3: wide field (+-79 deg),
//                                              4: wider than the table takes (+-86 deg)
// prints "ok <row decisions> <row settles> <col decisions> <col settles>" or "FAIL ...".
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "flic_internal.h"

int main(int argc, char** argv) {
    if (argc < 5) return 2;
    const int R = atoi(argv[1]), C = atoi(argv[2]);
    const unsigned seed = (unsigned)atoi(argv[3]);
    const long trials = atol(argv[4]);
    const int mode = argc > 5 ? atoi(argv[5]) : 0;
    std::mt19937_64 g(seed);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    const double kPi = 3.14159265358979323846;
    std::vector<double> elev(R);
    const double lo = mode == 2 ? -0.5 : (mode == 3 ? -79.0 : (mode == 4 ? -86.0 : -25.0));
    const double hi = mode == 2 ? 0.5 : (mode == 3 ? 79.0 : (mode == 4 ? 86.0 : 15.0));
    for (int r = 0; r < R; ++r)  // roughly even beams with jitter
        elev[r] = (lo + (hi - lo) * (r + 0.5 + 0.3 * (U(g) - 0.5)) / R) * kPi / 180.0;
    if (mode == 1)
        for (int r = R - 1; r > 0; --r) std::swap(elev[r], elev[g() % (r + 1)]);
    std::vector<float> colb(2 * C), rowb(2 * (R + 1));
    std::vector<int32_t> srow(R);
    std::vector<flic::RowSeed> seeds(flic::kRowSeeds);
    float t0 = 0, inv_dt = 0, margin = 0;
    const double az = 2 * kPi / C;
    if (!flic::build_proj_tables_into(R, C, elev.data(), az, colb.data(), rowb.data(),
                                      srow.data(), seeds.data(), &t0, &inv_dt, &margin)) {
        printf("FAIL builder refused\n");
        return 1;
    }
    // boundaries in double, as the builder defines them
    std::vector<double> sorted(R), bnd(R + 1);
    for (int j = 0; j < R; ++j) sorted[j] = elev[srow[j]];
    bnd[0] = sorted[0] - (sorted[1] - sorted[0]) / 2;
    bnd[R] = sorted[R - 1] + (sorted[R - 1] - sorted[R - 2]) / 2;
    for (int j = 1; j < R; ++j) bnd[j] = (sorted[j - 1] + sorted[j]) / 2;
    long rdec = 0, rset = 0, cdec = 0, cset = 0;
    const bool table = inv_dt > 0;
    for (long t = 0; t < trials && table; ++t) {
        // an elevation in or near the field, half of them close to a boundary
        double e;
        if (t & 1) {
            const int k = (int)(g() % (R + 1));
            e = bnd[k] + (U(g) < 0.5 ? -1 : 1) * std::pow(10.0, -9.0 + 6.0 * U(g));
        } else {
            e = bnd[0] - 0.01 + (bnd[R] - bnd[0] + 0.02) * U(g);
        }
        const double tt = std::tan(e);
        const double err = (2 * U(g) - 1) * 2.4e-7 * std::fabs(tt);
        const float tc = (float)(tt + err);
        const float fb = (tc - t0) * inv_dt;
        const int b = (int)std::fmin(std::fmax(fb, 0.0f), (float)(flic::kRowSeeds - 1));
        const flic::RowSeed& s = seeds[b];
        int row;
        if (tc < s.tlo) row = (int)((s.info >> 10) & 1023u);
        else if (tc > s.thi) row = (int)((s.info >> 20) & 1023u);
        else { ++rset; continue; }
        ++rdec;
        double dmin = 1e9;
        int band = -1;  // exact band: boundaries below e
        for (int k = 0; k <= R; ++k) {
            dmin = std::fmin(dmin, std::fabs(e - bnd[k]));
            if (bnd[k] <= e) band = k;
        }
        const int want = band < 0 || band >= R ? (int)flic::kRowOutside : srow[band];
        if (dmin <= 1e-6 || row != want) {
            printf("FAIL row e=%.12g dmin=%.3g bucket=%d got=%d want=%d\n", e, dmin, b, row, want);
            return 1;
        }
    }
    for (long t = 0; t < trials; ++t) {
        double phi;
        if (t & 1) {
            const int c = (int)(g() % C);
            phi = c * az + (U(g) < 0.5 ? -1 : 1) * std::pow(10.0, -9.0 + 6.0 * U(g));
            if (phi < 0) phi += 2 * kPi;
        } else {
            phi = 2 * kPi * U(g);
        }
        const double seedv = phi + (2 * U(g) - 1) * 1.1e-6;
        const float fc = (float)seedv * (float)(1.0 / az);
        int c = (int)fc;
        c = c < 0 ? 0 : (c >= C ? C - 1 : c);
        const float fr = fc - (float)c;
        if (!(fr > margin && fr < 1.0f - margin)) { ++cset; continue; }
        ++cdec;
        const int want = (int)std::floor(phi / az);
        const double d = std::fmin(std::fabs(phi - want * az), std::fabs(phi - (want + 1) * az));
        if (d <= 1e-6 || c != want % C) {
            printf("FAIL col phi=%.12g d=%.3g got=%d want=%d\n", phi, d, c, want);
            return 1;
        }
    }
    printf("ok %ld %ld %ld %ld %d\n", rdec, rset, cdec, cset, table ? 1 : 0);
    return 0;
}
