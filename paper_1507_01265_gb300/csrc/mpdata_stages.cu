// Stage-per-kernel MPDATA step: one kernel per stage, every intermediate in
// HBM.  This is the plain GPU formulation of the step (§5.2; the paper notes
// that running stage by stage through main memory is what makes MPDATA
// memory-bound), kept as the correctness baseline for the fused kernel and
// as the "stage-per-kernel" arm of the fused-vs-staged comparison.
//
// Stages (one thread per cell, x fastest):
//   donor      psi1 = psi - (1/h) sum_d (F_d(upper face) - F_d(lower face))
//   antidiff   V_d on every lower face (pseudo-velocities with cross terms)
//   limiter    beta_up / beta_dn from the local extrema of psi and psi1
//              (Listing 1, stage 8) and the in/out antidiffusive fluxes
//   vmon       V_d limited by beta (in place)
//   donor      psi^{n+1} = corrective upstream pass of psi1 with V
//
// With three passes the last four stages run again on the result psi2 of
// the first corrective pass, the pseudo-velocities now built from the
// limited velocities V of that pass (each pass estimates the error of the
// pass before it).  Options of this path only: the extrema set (psi^n and
// the corrected field, or the corrected field alone) and, for FP32 fields,
// FP64 accumulation of the limiter's flux sums and beta factors.
#include "mpdata_internal.cuh"

namespace mpdata {
namespace {

constexpr int kBlockX = 128;

struct Cell {
    int i, j, k;
};

__device__ __forceinline__ long long lin(const Grid &g, int i, int j, int k) {
    return ((long long)k * g.ny + j) * g.nx + i;
}

template <typename T>
__device__ __forceinline__ T at(const Grid &g, const T *f, int i, int j, int k) {
    return f[lin(g, cell_index(i, g.nx, g.per[0]), cell_index(j, g.ny, g.per[1]),
                 cell_index(k, g.nz, g.per[2]))];
}

// Face value of a field staggered on `axis` at the face whose index on that
// axis is the `axis` component of (i,j,k) (0..n); the other components are
// cell indices.  Lid faces (index 0 or n on a lid axis) are zero.
template <typename T>
__device__ __forceinline__ T face(const Grid &g, const T *u, int axis, int i, int j, int k) {
    int idx[3] = {i, j, k};
    const int n[3] = {g.nx, g.ny, g.nz};
    int f = idx[axis];
    if (!g.per[axis] && (f <= 0 || f >= n[axis])) return T(0);
    if (f >= n[axis]) f -= n[axis];
    if (f < 0) f += n[axis];
    idx[axis] = f;
    for (int d = 0; d < 3; ++d)
        if (d != axis) idx[d] = cell_index(idx[d], n[d], g.per[d]);
    return u[lin(g, idx[0], idx[1], idx[2])];
}

__device__ __forceinline__ bool this_cell(const Grid &g, Cell &c) {
    c.i = blockIdx.x * kBlockX + threadIdx.x;
    c.j = blockIdx.y;
    c.k = blockIdx.z;
    return c.i < g.nx;
}

template <typename T>
__global__ void k_donor(Grid g, const T *__restrict__ h, const T *__restrict__ psi,
                        const T *__restrict__ w1, const T *__restrict__ w2,
                        const T *__restrict__ w3, T *__restrict__ out) {
    Cell c;
    if (!this_cell(g, c)) return;
    const int i = c.i, j = c.j, k = c.k;
    T p = psi[lin(g, i, j, k)];
    T fxl = upstream_flux(face(g, w1, 0, i, j, k), at(g, psi, i - 1, j, k), p);
    T fxh = upstream_flux(face(g, w1, 0, i + 1, j, k), p, at(g, psi, i + 1, j, k));
    T fyl = upstream_flux(face(g, w2, 1, i, j, k), at(g, psi, i, j - 1, k), p);
    T fyh = upstream_flux(face(g, w2, 1, i, j + 1, k), p, at(g, psi, i, j + 1, k));
    T fzl = upstream_flux(face(g, w3, 2, i, j, k), at(g, psi, i, j, k - 1), p);
    T fzh = upstream_flux(face(g, w3, 2, i, j, k + 1), p, at(g, psi, i, j, k + 1));
    T div = (fxh - fxl) + (fyh - fyl) + (fzh - fzl);
    out[lin(g, i, j, k)] = p - div / h[lin(g, i, j, k)];
}

// Pseudo-velocity on the lower face along `axis` of cell (i,j,k):
//   V = (|U| - U^2/hbar) A - U (Ubar_a B_a + Ubar_b B_b) / hbar
// with a = axis+1, b = axis+2 (mod 3).
template <typename T>
__device__ T antidiff(const Grid &g, const T *h, const T *p1, const T *const u[3], T eps,
                      int axis, int i, int j, int k) {
    const int idx[3] = {i, j, k};
    if (!g.per[axis] && idx[axis] == 0) return T(0);
    int e[3] = {0, 0, 0};
    e[axis] = 1;
    T U = face(g, u[axis], axis, i, j, k);
    T pR = at(g, p1, i, j, k);
    T pL = at(g, p1, i - e[0], j - e[1], k - e[2]);
    T A = (pR - pL) / (pR + pL + eps);
    T cross = T(0);
#pragma unroll
    for (int t = 1; t <= 2; ++t) {
        int ax = (axis + t) % 3;
        int s[3] = {0, 0, 0};
        s[ax] = 1;
        T sp = at(g, p1, i + s[0], j + s[1], k + s[2]) +
               at(g, p1, i + s[0] - e[0], j + s[1] - e[1], k + s[2] - e[2]);
        T sm = at(g, p1, i - s[0], j - s[1], k - s[2]) +
               at(g, p1, i - s[0] - e[0], j - s[1] - e[1], k - s[2] - e[2]);
        T B = T(0.5) * (sp - sm) / (sp + sm + eps);
        T Ubar = T(0.25) * (face(g, u[ax], ax, i - e[0], j - e[1], k - e[2]) +
                            face(g, u[ax], ax, i, j, k) +
                            face(g, u[ax], ax, i - e[0] + s[0], j - e[1] + s[1], k - e[2] + s[2]) +
                            face(g, u[ax], ax, i + s[0], j + s[1], k + s[2]));
        cross = (t == 1) ? Ubar * B : cross + Ubar * B;
    }
    T hbar = T(0.5) * (at(g, h, i - e[0], j - e[1], k - e[2]) + at(g, h, i, j, k));
    return (fabs(U) - U * U / hbar) * A - U * cross / hbar;
}

template <typename T>
__global__ void k_antidiff(Grid g, T eps, const T *__restrict__ h, const T *__restrict__ p1,
                           const T *__restrict__ u1, const T *__restrict__ u2,
                           const T *__restrict__ u3, T *__restrict__ v1, T *__restrict__ v2,
                           T *__restrict__ v3) {
    Cell c;
    if (!this_cell(g, c)) return;
    const T *u[3] = {u1, u2, u3};
    long long q = lin(g, c.i, c.j, c.k);
    v1[q] = antidiff(g, h, p1, u, eps, 0, c.i, c.j, c.k);
    v2[q] = antidiff(g, h, p1, u, eps, 1, c.i, c.j, c.k);
    v3[q] = antidiff(g, h, p1, u, eps, 2, c.i, c.j, c.k);
}

// Limiter factors of the pass that corrects p: extrema over the 7-point
// stencil of p and (extrema == 0) psi^n; the in/out flux sums and the beta
// ratios are accumulated in Acc (T, or double for the FP64-beta option).
template <typename T, typename Acc>
__global__ void k_limiter(Grid g, Acc eps, int extrema, const T *__restrict__ h,
                          const T *__restrict__ psi, const T *__restrict__ p1,
                          const T *__restrict__ v1, const T *__restrict__ v2,
                          const T *__restrict__ v3, T *__restrict__ bup, T *__restrict__ bdn) {
    Cell c;
    if (!this_cell(g, c)) return;
    const int i = c.i, j = c.j, k = c.k;
    const int off[7][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0},
                           {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    T mx = at(g, p1, i, j, k), mn = mx;
#pragma unroll
    for (int n = 0; n < 7; ++n) {
        T b = at(g, p1, i + off[n][0], j + off[n][1], k + off[n][2]);
        mx = fmax(mx, b);
        mn = fmin(mn, b);
        if (extrema == 0) {
            T a = at(g, psi, i + off[n][0], j + off[n][1], k + off[n][2]);
            mx = fmax(mx, a);
            mn = fmin(mn, a);
        }
    }
    const T *v[3] = {v1, v2, v3};
    const T pc = at(g, p1, i, j, k);
    Acc in = Acc(0), out = Acc(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int e[3] = {0, 0, 0};
        e[d] = 1;
        const Acc vlo = face(g, v[d], d, i, j, k);
        const Acc vhi = face(g, v[d], d, i + e[0], j + e[1], k + e[2]);
        in += fmax(vlo, Acc(0)) * Acc(at(g, p1, i - e[0], j - e[1], k - e[2])) -
              fmin(vhi, Acc(0)) * Acc(at(g, p1, i + e[0], j + e[1], k + e[2]));
        out += fmax(vhi, Acc(0)) * Acc(pc) - fmin(vlo, Acc(0)) * Acc(pc);
    }
    const Acc hc = h[lin(g, i, j, k)];
    bup[lin(g, i, j, k)] = T((Acc(mx) - Acc(pc)) * hc / (in + eps));
    bdn[lin(g, i, j, k)] = T((Acc(pc) - Acc(mn)) * hc / (out + eps));
}

template <typename T>
__global__ void k_vmon(Grid g, const T *__restrict__ bup, const T *__restrict__ bdn,
                       T *__restrict__ v1, T *__restrict__ v2, T *__restrict__ v3) {
    Cell c;
    if (!this_cell(g, c)) return;
    const int i = c.i, j = c.j, k = c.k;
    T *v[3] = {v1, v2, v3};
    long long q = lin(g, i, j, k);
    T bu = bup[q], bd = bdn[q];
    const int idx[3] = {i, j, k};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (!g.per[d] && idx[d] == 0) {
            v[d][q] = T(0);
            continue;
        }
        int e[3] = {0, 0, 0};
        e[d] = 1;
        T buL = at(g, bup, i - e[0], j - e[1], k - e[2]);
        T bdL = at(g, bdn, i - e[0], j - e[1], k - e[2]);
        T V = v[d][q];
        v[d][q] = fmax(V, T(0)) * fmin(T(1), fmin(bdL, bu)) +
                  fmin(V, T(0)) * fmin(T(1), fmin(buL, bd));
    }
}

inline dim3 grid_of(const Grid &g) {
    return dim3((g.nx + kBlockX - 1) / kBlockX, g.ny, g.nz);
}

template <typename T>
cudaError_t donor_t(const Grid &g, const void *h, const void *psi, const void *w1, const void *w2,
                    const void *w3, void *out, cudaStream_t s) {
    k_donor<T><<<grid_of(g), kBlockX, 0, s>>>(g, (const T *)h, (const T *)psi, (const T *)w1,
                                               (const T *)w2, (const T *)w3, (T *)out);
    return cudaGetLastError();
}

// One corrective pass: antidiffusive velocities of the field p (made with
// the face velocities w) into v, limiter (in place on v), corrective donor
// pass of p with v into out.
template <typename T>
void corrective_pass_t(const Grid &g, int nonosc, int extrema, int precision, double eps,
                       const T *h, const T *psi, const T *p, const T *const w[3], T *const v[3],
                       T *bup, T *bdn, T *out, cudaStream_t s) {
    dim3 gr = grid_of(g);
    k_antidiff<T><<<gr, kBlockX, 0, s>>>(g, (T)eps, h, p, w[0], w[1], w[2], v[0], v[1], v[2]);
    if (nonosc) {
        if (precision == MPDATA_PREC_F64_BETA)
            k_limiter<T, double><<<gr, kBlockX, 0, s>>>(g, eps, extrema, h, psi, p, v[0], v[1],
                                                        v[2], bup, bdn);
        else
            k_limiter<T, T><<<gr, kBlockX, 0, s>>>(g, (T)eps, extrema, h, psi, p, v[0], v[1], v[2],
                                                   bup, bdn);
        k_vmon<T><<<gr, kBlockX, 0, s>>>(g, bup, bdn, v[0], v[1], v[2]);
    }
    k_donor<T><<<gr, kBlockX, 0, s>>>(g, h, p, v[0], v[1], v[2], out);
}

template <typename T>
cudaError_t stage_step_t(const Grid &g, int iterations, int nonosc, int extrema, int precision,
                         double eps, const void *h, const void *psi, const void *u1,
                         const void *u2, const void *u3, void *out, const StageBuffers &b,
                         cudaStream_t s) {
    if (iterations <= 1) return donor_t<T>(g, h, psi, u1, u2, u3, out, s);
    dim3 gr = grid_of(g);
    const T *H = (const T *)h, *P = (const T *)psi;
    k_donor<T><<<gr, kBlockX, 0, s>>>(g, H, P, (const T *)u1, (const T *)u2, (const T *)u3,
                                       (T *)b.psi1);
    const T *const w[3] = {(const T *)u1, (const T *)u2, (const T *)u3};
    T *const v[3] = {(T *)b.v1, (T *)b.v2, (T *)b.v3};
    T *pass2 = iterations == 2 ? (T *)out : (T *)b.psi2;
    corrective_pass_t<T>(g, nonosc, extrema, precision, eps, H, P, (const T *)b.psi1, w, v,
                         (T *)b.bup, (T *)b.bdn, pass2, s);
    if (iterations == 3) {
        const T *const wv[3] = {v[0], v[1], v[2]};
        T *const v3[3] = {(T *)b.w1, (T *)b.w2, (T *)b.w3};
        corrective_pass_t<T>(g, nonosc, extrema, precision, eps, H, P, (const T *)b.psi2, wv, v3,
                             (T *)b.bup, (T *)b.bdn, (T *)out, s);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_donor(int dtype, const Grid &g, const void *h, const void *psi, const void *w1,
                         const void *w2, const void *w3, void *out, cudaStream_t s) {
    return dtype == MPDATA_F64 ? donor_t<double>(g, h, psi, w1, w2, w3, out, s)
                               : donor_t<float>(g, h, psi, w1, w2, w3, out, s);
}

cudaError_t launch_stage_step(int dtype, const Grid &g, int iterations, int nonosc, int extrema,
                              int precision, double eps, const void *h, const void *psi,
                              const void *u1, const void *u2, const void *u3, void *out,
                              const StageBuffers &b, cudaStream_t s) {
    return dtype == MPDATA_F64
               ? stage_step_t<double>(g, iterations, nonosc, extrema, precision, eps, h, psi, u1,
                                      u2, u3, out, b, s)
               : stage_step_t<float>(g, iterations, nonosc, extrema, precision, eps, h, psi, u1,
                                     u2, u3, out, b, s);
}

}  // namespace mpdata
