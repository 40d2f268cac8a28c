/*
 * mpdata_oracle.c -- serial FP64 reference of one 3D MPDATA time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only tests/, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py may load it.  It shares no code, header, table or helper
 * with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes (the paper, §5.2, names MPDATA as a nonoscillatory,
 * forward-in-time scheme built on upstream differencing and refers to the
 * published scheme for its equations; a step reads 5 matrices and returns 1):
 *
 *   (a1) donor-cell (upstream) pass           -> psi1
 *   (a2) antidiffusive pseudo-velocities      -> V1, V2, V3 (with cross terms)
 *   (a3) local extrema of psi^n and psi1      -> psimax, psimin (Listing 1,
 *        "stage 8": max over a cell and its 6 face neighbours)
 *   (a4) limiter factors                      -> beta_up, beta_dn
 *   (a5) limited velocities                   -> Vmon
 *   (a6) corrective donor-cell pass           -> psi^{n+1}
 *
 * With iterations = 3 stages (a2)-(a6) run a second time on the result of
 * the first corrective pass, the pseudo-velocities now built from the
 * limited velocities that pass used in place of the Courant numbers.  Each
 * corrective pass estimates the truncation error of the pass before it
 * (Smolarkiewicz 1984, §3, the iterated scheme), and under the
 * nonoscillatory option every iteration's pseudo-velocity is limited before
 * it transports anything (Smolarkiewicz & Grabowski 1990, §3): the pass
 * before the second corrective one is therefore the limited transport, and
 * its velocities are the limited ones.  Parity unpinned: that the second
 * pass is built from the limited (not the raw) velocities of the first is
 * this reading of Smolarkiewicz & Grabowski (1990), §3; no pin separates the
 * two (they coincide without the limiter).
 *
 * The formulas follow the published MPDATA scheme: the basic two-pass scheme
 * with its cross terms (Smolarkiewicz 1984, J. Comput. Phys. 54), the
 * nonoscillatory option (Smolarkiewicz & Grabowski 1990, J. Comput. Phys. 86)
 * and the form with a density/Jacobian h (Smolarkiewicz & Margolin 1998,
 * J. Comput. Phys. 140).  Each stage is a plain loop over every cell (or
 * face) into a full-size array, evaluated in the order the scheme states,
 * with no fusion, no blocking and no reordering.
 *
 * Conventions (the paper states none; these are the readings used):
 *   - arrays are [nz][ny][nx], x fastest; index (k*ny + j)*nx + i;
 *   - u1[k][j][i] is the Courant number on the x-face between cells i-1 and
 *     i (the lower x-face of cell i); u2, u3 likewise for y and z;
 *   - periodic axis: face 0 is the face between cells n-1 and 0;
 *   - lid axis: faces 0 and n carry zero velocity (the stored face-0 value
 *     is not read); ghost cells beyond a lid are zero-gradient copies of the
 *     edge cell (used by the cross terms and the extrema);
 *   - h-bar on a face is the mean of the two adjacent h;
 *   - eps is added to every A, B and beta denominator;
 *   - the extrema of a corrective pass are taken over psi^n and the field
 *     that pass corrects (psi1 for the first one), or, with extrema = 1,
 *     over the corrected field alone.
 *
 * An OpenMP build of this same file (-fopenmp) runs the per-cell loops on
 * all host cores; every cell is computed by the same expression as in the
 * serial build, so the two builds return identical bits.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    int periodic[3];     /* per axis: 1 periodic, 0 rigid lid */
    int iterations;      /* 1: donor cell only; 2, 3: one or two corrective passes */
    int nonoscillatory;  /* 1: apply the beta limiter to the antidiffusive velocities */
    double eps;          /* > 0 */
    int extrema;         /* 0: psi^n and the corrected field; 1: the corrected field only */
} oracle_cfg;

/* Optional intermediate outputs of the first corrective pass (any pointer
 * may be NULL). */
typedef struct {
    double *psi1;
    double *v1, *v2, *v3;
    double *beta_up, *beta_dn;
    double *vm1, *vm2, *vm3;
} oracle_stages;

static int dim_of(const oracle_cfg *c, int axis)
{
    return axis == 0 ? c->nx : (axis == 1 ? c->ny : c->nz);
}

/* Map a cell index on one axis into range: wrap on a periodic axis, clamp
 * (zero-gradient ghost) on a lid axis. */
static int cell_index(const oracle_cfg *c, int axis, int a)
{
    int n = dim_of(c, axis);
    if (a >= 0 && a < n) return a;
    if (c->periodic[axis]) {
        a %= n;
        if (a < 0) a += n;
        return a;
    }
    if (a < 0) return 0;
    if (a >= n) return n - 1;
    return a;
}

static long lin(const oracle_cfg *c, int i, int j, int k)
{
    return ((long)k * c->ny + j) * (long)c->nx + i;
}

/* Cell value with ghost rules applied on every axis. */
static double at(const oracle_cfg *c, const double *f, int i, int j, int k)
{
    return f[lin(c, cell_index(c, 0, i), cell_index(c, 1, j), cell_index(c, 2, k))];
}

/* Value of a face-staggered field of axis `axis` at the face whose index on
 * that axis is the `axis` component of (i,j,k) (0..n), the other two being
 * cell indices.  Lid faces (index 0 or n on a lid axis) are zero. */
static double face(const oracle_cfg *c, const double *u, int axis, int i, int j, int k)
{
    int idx[3] = {i, j, k};
    int n = dim_of(c, axis);
    int f = idx[axis];
    if (!c->periodic[axis] && (f <= 0 || f >= n)) return 0.0;
    if (f < 0 || f >= n) idx[axis] = ((f % n) + n) % n;
    for (int d = 0; d < 3; ++d)
        if (d != axis) idx[d] = cell_index(c, d, idx[d]);
    return u[lin(c, idx[0], idx[1], idx[2])];
}

/* Upstream flux through a face with velocity U between left cell value L
 * and right cell value R: [U]+ L + [U]- R. */
static double upstream_flux(double U, double L, double R)
{
    return fmax(U, 0.0) * L + fmin(U, 0.0) * R;
}

/* (a1)/(a6): one donor-cell pass of psi with face velocities w1, w2, w3:
 * out = psi - (1/h) * sum_d (F_d(upper face) - F_d(lower face)). */
static void donor_pass(const oracle_cfg *c, const double *h, const double *psi,
                       const double *w1, const double *w2, const double *w3, double *out)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                double p = at(c, psi, i, j, k);
                double fx_lo = upstream_flux(face(c, w1, 0, i, j, k), at(c, psi, i - 1, j, k), p);
                double fx_hi = upstream_flux(face(c, w1, 0, i + 1, j, k), p, at(c, psi, i + 1, j, k));
                double fy_lo = upstream_flux(face(c, w2, 1, i, j, k), at(c, psi, i, j - 1, k), p);
                double fy_hi = upstream_flux(face(c, w2, 1, i, j + 1, k), p, at(c, psi, i, j + 1, k));
                double fz_lo = upstream_flux(face(c, w3, 2, i, j, k), at(c, psi, i, j, k - 1), p);
                double fz_hi = upstream_flux(face(c, w3, 2, i, j, k + 1), p, at(c, psi, i, j, k + 1));
                double div = (fx_hi - fx_lo) + (fy_hi - fy_lo) + (fz_hi - fz_lo);
                out[lin(c, i, j, k)] = p - div / at(c, h, i, j, k);
            }
}

/* (a2): antidiffusive pseudo-velocity on the lower face (along `axis`) of
 * cell (i,j,k), for the field psi1 being corrected and the face velocities
 * u of the pass that made it.  With e the unit step along `axis` and a, b
 * the two other axes:
 *   A   = (psi1[c] - psi1[c-e]) / (psi1[c] + psi1[c-e] + eps)
 *   B_a = 1/2 (S(c+e_a) - S(c-e_a)) / (S(c+e_a) + S(c-e_a) + eps),
 *         S(x) = psi1[x] + psi1[x-e]            (the pair across the face)
 *   Ubar_a = 1/4 (u_a at the 4 a-faces touching the two cells of the pair)
 *   hbar = (h[c-e] + h[c]) / 2
 *   V = (|U| - U^2/hbar) A - U (Ubar_a B_a + Ubar_b B_b) / hbar          */
static double antidiffusive_velocity(const oracle_cfg *c, const double *h, const double *psi1,
                                     const double *u[3], int axis, int i, int j, int k)
{
    int idx[3] = {i, j, k};
    if (!c->periodic[axis] && idx[axis] == 0) return 0.0;   /* lid face */
    int e[3] = {0, 0, 0};
    e[axis] = 1;
    int a = (axis + 1) % 3, b = (axis + 2) % 3;
    int ea[3] = {0, 0, 0}, eb[3] = {0, 0, 0};
    ea[a] = 1;
    eb[b] = 1;

    double U = face(c, u[axis], axis, i, j, k);
    double pR = at(c, psi1, i, j, k);
    double pL = at(c, psi1, i - e[0], j - e[1], k - e[2]);
    double A = (pR - pL) / (pR + pL + c->eps);

    double B[2], Ubar[2];
    int other[2] = {a, b};
    for (int t = 0; t < 2; ++t) {
        int *s = (t == 0) ? ea : eb;
        int ax = other[t];
        double sp = at(c, psi1, i + s[0], j + s[1], k + s[2]) +
                    at(c, psi1, i + s[0] - e[0], j + s[1] - e[1], k + s[2] - e[2]);
        double sm = at(c, psi1, i - s[0], j - s[1], k - s[2]) +
                    at(c, psi1, i - s[0] - e[0], j - s[1] - e[1], k - s[2] - e[2]);
        B[t] = 0.5 * (sp - sm) / (sp + sm + c->eps);
        /* the four faces of axis ax around the pair (c-e, c): lower and
         * upper ax-face of each of the two cells */
        Ubar[t] = 0.25 * (face(c, u[ax], ax, i - e[0], j - e[1], k - e[2]) +
                          face(c, u[ax], ax, i, j, k) +
                          face(c, u[ax], ax, i - e[0] + s[0], j - e[1] + s[1], k - e[2] + s[2]) +
                          face(c, u[ax], ax, i + s[0], j + s[1], k + s[2]));
    }
    double hbar = 0.5 * (at(c, h, i - e[0], j - e[1], k - e[2]) + at(c, h, i, j, k));
    return (fabs(U) - U * U / hbar) * A - U * (Ubar[0] * B[0] + Ubar[1] * B[1]) / hbar;
}

/* (a3): maximum (sign=+1) or minimum (sign=-1) over the cell and its six
 * face neighbours (Listing 1, stage 8) of the corrected field p and, unless
 * c->extrema is 1, of psi^n. */
static double local_extremum(const oracle_cfg *c, const double *psi, const double *p,
                             int i, int j, int k, int sign)
{
    static const int off[7][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0},
                                  {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    double m = at(c, p, i, j, k);
    for (int n = 0; n < 7; ++n) {
        double b = at(c, p, i + off[n][0], j + off[n][1], k + off[n][2]);
        m = sign > 0 ? fmax(m, b) : fmin(m, b);
        if (c->extrema == 0) {
            double a = at(c, psi, i + off[n][0], j + off[n][1], k + off[n][2]);
            m = sign > 0 ? fmax(m, a) : fmin(m, a);
        }
    }
    return m;
}

/* One corrective pass (a2)-(a6): the field p (the result of the pass before)
 * is corrected with pseudo-velocities built from p and the face velocities
 * w that the pass before used.  v receives the pseudo-velocities, vm the
 * velocities this pass transports with (v limited, or v itself), next the
 * corrected field.  bup/bdn are work arrays. */
static void corrective_pass(const oracle_cfg *c, const double *h, const double *psi,
                            const double *p, const double *w[3], double *v[3], double *vm[3],
                            double *bup, double *bdn, double *next)
{
    long n = (long)c->nx * c->ny * c->nz;

    /* (a2) antidiffusive pseudo-velocities on every lower face */
    for (int d = 0; d < 3; ++d) {
        double *vd = v[d];
#pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < c->nz; ++k)
            for (int j = 0; j < c->ny; ++j)
                for (int i = 0; i < c->nx; ++i)
                    vd[lin(c, i, j, k)] = antidiffusive_velocity(c, h, p, w, d, i, j, k);
    }

    if (c->nonoscillatory) {
        /* (a3) + (a4): extrema and limiter factors per cell */
#pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < c->nz; ++k)
            for (int j = 0; j < c->ny; ++j)
                for (int i = 0; i < c->nx; ++i) {
                    double mx = local_extremum(c, psi, p, i, j, k, +1);
                    double mn = local_extremum(c, psi, p, i, j, k, -1);
                    double pc = at(c, p, i, j, k);
                    double in = 0.0, outf = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        int e[3] = {0, 0, 0};
                        e[d] = 1;
                        double vlo = face(c, v[d], d, i, j, k);
                        double vhi = face(c, v[d], d, i + e[0], j + e[1], k + e[2]);
                        in += fmax(vlo, 0.0) * at(c, p, i - e[0], j - e[1], k - e[2]) -
                              fmin(vhi, 0.0) * at(c, p, i + e[0], j + e[1], k + e[2]);
                        outf += fmax(vhi, 0.0) * pc - fmin(vlo, 0.0) * pc;
                    }
                    double hc = at(c, h, i, j, k);
                    bup[lin(c, i, j, k)] = (mx - pc) * hc / (in + c->eps);
                    bdn[lin(c, i, j, k)] = (pc - mn) * hc / (outf + c->eps);
                }
        /* (a5): limited velocities on every lower face, between L = c-e and R = c */
        for (int d = 0; d < 3; ++d) {
            double *vd = v[d], *vmd = vm[d];
#pragma omp parallel for collapse(2) schedule(static)
            for (int k = 0; k < c->nz; ++k)
                for (int j = 0; j < c->ny; ++j)
                    for (int i = 0; i < c->nx; ++i) {
                        int idx[3] = {i, j, k};
                        long cR = lin(c, i, j, k);
                        if (!c->periodic[d] && idx[d] == 0) { vmd[cR] = 0.0; continue; }
                        int e[3] = {0, 0, 0};
                        e[d] = 1;
                        double bupL = at(c, bup, i - e[0], j - e[1], k - e[2]);
                        double bdnL = at(c, bdn, i - e[0], j - e[1], k - e[2]);
                        double V = vd[cR];
                        vmd[cR] = fmax(V, 0.0) * fmin(1.0, fmin(bdnL, bup[cR])) +
                                  fmin(V, 0.0) * fmin(1.0, fmin(bupL, bdn[cR]));
                    }
        }
    } else {
        for (int d = 0; d < 3; ++d) memcpy(vm[d], v[d], sizeof(double) * n);
    }

    /* (a6) corrective donor-cell pass of p with the (limited) velocities */
    donor_pass(c, h, p, vm[0], vm[1], vm[2], next);
}

static int run_step(const oracle_cfg *c, const double *h, const double *psi,
                    const double *u1, const double *u2, const double *u3,
                    double *out, oracle_stages *st)
{
    long n = (long)c->nx * c->ny * c->nz;
    /* work arrays: psi1, the field after pass 2, V[3], Vmon[3], the
     * velocities of the pass before [3], beta_up, beta_dn */
    enum { NWORK = 13 };
    double *wk[NWORK];
    int nwork = c->iterations <= 1 ? 1 : NWORK;
    for (int a = 0; a < NWORK; ++a) wk[a] = NULL;
    for (int a = 0; a < nwork; ++a) {
        wk[a] = malloc(sizeof(double) * n);
        if (!wk[a]) {
            for (int b = 0; b < a; ++b) free(wk[b]);
            return -1;
        }
    }
    double *psi1 = wk[0], *psi2 = wk[1];
    double *v[3] = {wk[2], wk[3], wk[4]}, *vm[3] = {wk[5], wk[6], wk[7]};
    double *wprev[3] = {wk[8], wk[9], wk[10]};
    double *bup = wk[11], *bdn = wk[12];

    /* (a1) donor-cell pass */
    donor_pass(c, h, psi, u1, u2, u3, psi1);
    if (st && st->psi1) memcpy(st->psi1, psi1, sizeof(double) * n);
    if (c->iterations <= 1) {
        memcpy(out, psi1, sizeof(double) * n);
        free(psi1);
        return 0;
    }

    /* first corrective pass: psi1 corrected, pseudo-velocities from U */
    const double *w[3] = {u1, u2, u3};
    double *next = c->iterations == 2 ? out : psi2;
    corrective_pass(c, h, psi, psi1, w, v, vm, bup, bdn, next);
    if (st) {
        double **dst_v[3] = {&st->v1, &st->v2, &st->v3};
        double **dst_m[3] = {&st->vm1, &st->vm2, &st->vm3};
        for (int d = 0; d < 3; ++d) {
            if (*dst_v[d]) memcpy(*dst_v[d], v[d], sizeof(double) * n);
            if (*dst_m[d]) memcpy(*dst_m[d], vm[d], sizeof(double) * n);
        }
        if (st->beta_up) {
            if (c->nonoscillatory) memcpy(st->beta_up, bup, sizeof(double) * n);
            else memset(st->beta_up, 0, sizeof(double) * n);
        }
        if (st->beta_dn) {
            if (c->nonoscillatory) memcpy(st->beta_dn, bdn, sizeof(double) * n);
            else memset(st->beta_dn, 0, sizeof(double) * n);
        }
    }

    if (c->iterations == 3) {
        /* second corrective pass: psi2 corrected, pseudo-velocities built
         * from the velocities the first corrective pass transported with
         * (the limited ones under the nonoscillatory option: Smolarkiewicz &
         * Grabowski 1990, §3, limit every iteration before it transports) */
        for (int d = 0; d < 3; ++d) memcpy(wprev[d], vm[d], sizeof(double) * n);
        const double *w2[3] = {wprev[0], wprev[1], wprev[2]};
        corrective_pass(c, h, psi, psi2, w2, v, vm, bup, bdn, out);
    }

    for (int a = 0; a < nwork; ++a) free(wk[a]);
    return 0;
}

static int cfg_ok(const oracle_cfg *c)
{
    if (!c || c->nx <= 0 || c->ny <= 0 || c->nz <= 0) return 0;
    if (c->iterations < 1 || c->iterations > 3) return 0;
    if (c->extrema != 0 && c->extrema != 1) return 0;
    if (!(c->eps > 0.0)) return 0;
    return 1;
}

/* One step: psi_out = MPDATA(psi).  psi_out must not alias psi.
 * Returns 0, or -1 on invalid configuration / allocation failure. */
int oracle_step(const oracle_cfg *c, const double *h, const double *psi, const double *u1,
                const double *u2, const double *u3, double *psi_out, oracle_stages *st)
{
    if (!cfg_ok(c) || psi == psi_out) return -1;
    return run_step(c, h, psi, u1, u2, u3, psi_out, st);
}

/* nsteps steps in place on psi. */
int oracle_run(const oracle_cfg *c, const double *h, double *psi, const double *u1,
               const double *u2, const double *u3, int nsteps)
{
    if (!cfg_ok(c) || nsteps < 0) return -1;
    long n = (long)c->nx * c->ny * c->nz;
    double *tmp = malloc(sizeof(double) * n);
    if (!tmp) return -1;
    for (int s = 0; s < nsteps; ++s) {
        if (run_step(c, h, psi, u1, u2, u3, tmp, NULL)) { free(tmp); return -1; }
        memcpy(psi, tmp, sizeof(double) * n);
    }
    free(tmp);
    return 0;
}

/* (a8) total mass sum h*psi, accumulated with Neumaier's compensated
 * summation so that the sum itself adds no error at the 1e-12 level. */
double oracle_mass(long n, const double *h, const double *psi)
{
    double s = 0.0, comp = 0.0;
    for (long q = 0; q < n; ++q) {
        double x = h[q] * psi[q];
        double t = s + x;
        if (fabs(s) >= fabs(x)) comp += (s - t) + x;
        else comp += (x - t) + s;
        s = t;
    }
    return s + comp;
}

/* Number of threads the per-cell loops use (1 in the serial build). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
