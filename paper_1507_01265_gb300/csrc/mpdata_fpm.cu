// Functional-performance-model partitioning (§2, §3, Algorithm 1 of §4).
//
// A speed function s(x) gives the speed (work units per second) of one
// processor executing a workload of size x while all processors run
// (measured under contention, §5.4).  The execution time of x is x / s(x).
// Algorithm 1 distributes n units over p identical processors, each taking a
// multiple of dx, so that the largest execution time is minimal: starting
// from the balanced share n/p it moves dx from "left" processors to "right"
// processors step by step and keeps the best (x_left, x_right); p/2
// processors get each size.  The printed loop bound ("until x_r < n") would
// stop after one pass; it is read as "while x_left - dx stays positive".
// The strict "t < t_min" keeps the first minimum.
//
// The general form (any p, P:"easily generalised") lets k of the p
// processors take x_right = n/p + j dx and the other p - k share the rest
// equally, x_left = (n - k x_right) / (p - k), kept only when x_left is a
// positive multiple of dx; j = 0 is the balanced split.
//
// s(x) is a table of measured points, linearly interpolated; sizes outside
// the table are not considered.
#include <math.h>

#include "mpdata_internal.cuh"

namespace {

bool speed_at(const double *xs, const double *ss, int npts, double x, double *s) {
    if (npts < 1 || x < xs[0] - 1e-9 || x > xs[npts - 1] + 1e-9) return false;
    if (npts == 1) { *s = ss[0]; return true; }
    int i = 0;
    while (i < npts - 2 && x > xs[i + 1]) ++i;
    const double w = (xs[i + 1] == xs[i]) ? 0.0 : (x - xs[i]) / (xs[i + 1] - xs[i]);
    *s = ss[i] + w * (ss[i + 1] - ss[i]);
    return *s > 0.0;
}

bool time_of(const double *xs, const double *ss, int npts, double x, double *t) {
    double s;
    if (!speed_at(xs, ss, npts, x, &s)) return false;
    *t = x / s;
    return true;
}

bool on_grid(double x, double dx) {
    const double q = x / dx;
    return fabs(q - nearbyint(q)) < 1e-9 * (1.0 + fabs(q));
}

int check_table(const double *xs, const double *ss, int npts) {
    if (!xs || !ss || npts < 1) return mpdata::set_error(MPDATA_EINVAL, "speed table is empty");
    for (int i = 0; i < npts; ++i) {
        if (!(ss[i] > 0.0)) return mpdata::set_error(MPDATA_EINVAL, "speeds must be > 0");
        if (i && !(xs[i] > xs[i - 1])) return mpdata::set_error(MPDATA_EINVAL, "sizes must increase");
    }
    return MPDATA_OK;
}

}  // namespace

extern "C" {

int mpdata_fpm_algorithm1(double n, int p, double dx, const double *xs, const double *ss, int npts,
                          double *x_left, double *x_right, double *t_min) {
    if (!x_left || !x_right || !t_min) return mpdata::set_error(MPDATA_EINVAL, "NULL output");
    if (!(n > 0) || p < 2 || (p & 1) || !(dx > 0)) return mpdata::set_error(MPDATA_EINVAL, "Algorithm 1 needs n > 0, even p >= 2, dx > 0");
    int rc = check_table(xs, ss, npts);
    if (rc) return rc;
    const double share = n / p;
    if (!on_grid(share, dx)) return mpdata::set_error(MPDATA_EINVAL, "n/p must be a multiple of dx");
    double xr = share, xl = share, t;
    if (!time_of(xs, ss, npts, share, &t)) return mpdata::set_error(MPDATA_EINVAL, "n/p is outside the speed table");
    double best = t, br = xr, bl = xl;
    while (xl - dx > 0) {
        xr += dx;
        xl -= dx;
        double tr, tl;
        if (!time_of(xs, ss, npts, xr, &tr) || !time_of(xs, ss, npts, xl, &tl)) break;
        t = tr > tl ? tr : tl;
        if (t < best) { best = t; br = xr; bl = xl; }
    }
    *x_left = bl;
    *x_right = br;
    *t_min = best;
    return MPDATA_OK;
}

int mpdata_fpm_partition(double n, int p, double dx, const double *xs, const double *ss, int npts,
                         int *k_right, double *x_left, double *x_right, double *t_min) {
    if (!k_right || !x_left || !x_right || !t_min) return mpdata::set_error(MPDATA_EINVAL, "NULL output");
    if (!(n > 0) || p < 1 || !(dx > 0)) return mpdata::set_error(MPDATA_EINVAL, "need n > 0, p >= 1, dx > 0");
    int rc = check_table(xs, ss, npts);
    if (rc) return rc;
    const double share = n / p;
    // balanced reference: every processor takes n/p (or, off the dx grid,
    // the nearest two-size split found below with j = 0 equivalent)
    double best = INFINITY, br = share, bl = share;
    int bk = 0;
    double t;
    if (on_grid(share, dx) && time_of(xs, ss, npts, share, &t)) { best = t; bk = 0; }
    for (int k = 1; k < p; ++k) {
        // smallest x_right on the dx grid that is >= n/p
        double xr = ceil(share / dx - 1e-9) * dx;
        for (;; xr += dx) {
            const double rem = n - k * xr;
            if (rem <= 0) break;
            const double xl = rem / (p - k);
            if (xl < dx - 1e-9 * dx) break;
            if (!on_grid(xl, dx)) continue;
            double tr, tl;
            if (!time_of(xs, ss, npts, xr, &tr)) break;
            if (!time_of(xs, ss, npts, xl, &tl)) continue;
            t = tr > tl ? tr : tl;
            if (t < best) { best = t; br = xr; bl = xl; bk = k; }
        }
    }
    if (!isfinite(best)) return mpdata::set_error(MPDATA_EINVAL, "no split of n fits the speed table");
    *k_right = bk;
    *x_left = bl;
    *x_right = br;
    *t_min = best;
    return MPDATA_OK;
}

int mpdata_fpm_condition2(const double *xs, const double *ss, int npts, double *x_at, double *x_more) {
    // condition (2) of §3: exists x < x' with s(x)/x < s(x')/x' (a larger
    // workload finishes no later), i.e. load balancing is not guaranteed optimal
    int rc = check_table(xs, ss, npts);
    if (rc) return rc < 0 ? rc : -1;
    for (int i = 0; i < npts; ++i)
        for (int j = i + 1; j < npts; ++j)
            if (ss[i] / xs[i] < ss[j] / xs[j]) {
                if (x_at) *x_at = xs[i];
                if (x_more) *x_more = xs[j];
                return 1;
            }
    return 0;
}

}  // extern "C"
