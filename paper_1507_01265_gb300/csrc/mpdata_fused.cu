// Fused MPDATA step: every stage of one time step in one kernel (§5.2's
// dependent stencil stages; the paper's (3+1)D decomposition in §5.3 keeps
// the intermediates of a block in cache -- here they live in shared memory
// and registers, so a step moves only the 5 input fields and the output
// through HBM).
//
// Decomposition (GB300-first, not the Xeon Phi code):
//   * a CTA owns an output tile of TX x TY columns and marches it through all
//     z planes; every quantity a column needs from its own z-neighbours is
//     carried in registers, x/y neighbours go through shared-memory planes;
//   * each stage is evaluated on exactly the columns later stages need
//     (psi1 on radius 2, pseudo-velocities on radius ~1.5, limiter factors on
//     radius 1, limited fluxes on radius 0..1).  Thread t owns one column and
//     columns are numbered from the tile outwards ring by ring, so a stage's
//     region is a prefix of the thread index and idle threads are whole warps;
//   * inputs (psi, u1, u2, u3, h) of radius 3 stream into a 4-plane
//     shared-memory ring with cp.async one plane ahead of use; the zero-fill
//     form of cp.async supplies the zero velocity of lid faces;
//   * per plane p: donor pass at p-1 | pseudo-velocities of the x/y faces at
//     p-2 | z-face pseudo-velocity above p-2 and limiter factors at p-2 |
//     limited corrective fluxes at p-2 and the finished output at p-3.
//
// Boundary rules (the oracle's readings): periodic axes wrap; on a lid axis
// faces 0 and n carry zero velocity and ghost cells are zero-gradient copies
// (clamped neighbour reads in x/y, copied queue entries in z).
//
// Arithmetic: FP32 divisions are a hardware reciprocal (rcp.approx, <= 1 ulp)
// times the numerator, one reciprocal per denominator; FP64 keeps IEEE
// reciprocals.  Local extrema use the 3-input min/max of sm_100+.
#include <algorithm>
#include <map>

#include "mpdata_internal.cuh"

namespace mpdata {
namespace {

template <int TX, int TY>
struct Layout {
    static constexpr int EX = TX + 6, EY = TY + 6, PL = EX * EY;  // radius-3 plane
    static constexpr int NT = (TX + 4) * (TY + 4);                 // psi1 region = threads
    static constexpr int N_OUT = TX * TY;
    static constexpr int N_VM = (TX + 1) * (TY + 1);
    static constexpr int N_BETA = (TX + 2) * (TY + 2);
    static constexpr int N_V = (TX + 3) * (TY + 3);
    // plane buffers (each PL elements)
    static constexpr int RING = 0;    // 5 fields x 4 planes
    static constexpr int P1 = 20;     // psi1, 2 planes
    static constexpr int SX = 22;     // x-pair sums, 2 planes
    static constexpr int SY = 24;     // y-pair sums, 2 planes
    static constexpr int SZ = 26;     // z-pair sums of the face above q2
    static constexpr int V1 = 27, V2 = 28, BU = 29, BD = 30, GX = 31, GY = 32;
    static constexpr int NPLANES = 33;
    static_assert(PL <= 2 * NT, "each thread loads at most two columns");
};

// Column of thread t relative to the tile origin, rings numbered outwards:
// [0, TX)x[0, TY) | +col TX, +row TY | row -1, col -1 | col TX+1, row TY+1 |
// row -2, col -2.
template <int TX, int TY>
__device__ __forceinline__ void onion(int t, int &rx, int &ry) {
    if (t < TX * TY) { rx = t % TX; ry = t / TX; return; }
    t -= TX * TY;
    if (t < TY + 1) { rx = TX; ry = t; return; }
    t -= TY + 1;
    if (t < TX) { rx = t; ry = TY; return; }
    t -= TX;
    if (t < TX + 2) { rx = t - 1; ry = -1; return; }
    t -= TX + 2;
    if (t < TY + 1) { rx = -1; ry = t; return; }
    t -= TY + 1;
    if (t < TY + 3) { rx = TX + 1; ry = t - 1; return; }
    t -= TY + 3;
    if (t < TX + 2) { rx = t - 1; ry = TY + 1; return; }
    t -= TX + 2;
    if (t < TX + 4) { rx = t - 2; ry = -2; return; }
    t -= TX + 4;
    rx = -2;
    ry = t - 1;
}

__device__ __forceinline__ int wrap_or_clamp(int a, int n, int per) {
    if (a >= 0 && a < n) return a;
    if (per) { a %= n; return a < 0 ? a + n : a; }
    return a < 0 ? 0 : n - 1;
}

template <typename T>
__device__ __forceinline__ void cp_async(unsigned dst, const T *src, bool zero) {
    int bytes = zero ? 0 : (int)sizeof(T);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(src),
                 "n"(sizeof(T)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Reciprocal: FP32 hardware approximation (<= 1 ulp), FP64 IEEE.
__device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

__device__ __forceinline__ float max3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ double max3(double a, double b, double c) { return fmax(fmax(a, b), c); }
__device__ __forceinline__ double min3(double a, double b, double c) { return fmin(fmin(a, b), c); }

template <typename T>
__device__ __forceinline__ T pos(T a) { return a > T(0) ? a : T(0); }
template <typename T>
__device__ __forceinline__ T neg(T a) { return a < T(0) ? a : T(0); }

// Pseudo-velocity on a face from its pieces (pair sums s* across the face,
// sums of the 4 transverse face velocities u*, h-sum of the two cells):
//   V = (|U| - U^2/hbar) A - U (Ubar_a B_a + Ubar_b B_b) / hbar
//   A = (pR - pL)/(pR + pL + eps), B = 1/2 (sp - sm)/(sp + sm + eps),
//   Ubar = usum/4, hbar = hsum/2.
template <typename T>
__device__ __forceinline__ T pseudo_velocity(T U, T pR, T pL, T spa, T sma, T ua, T spb, T smb,
                                             T ub, T hsum, T eps) {
    T A = (pR - pL) * rcp(pR + pL + eps);
    T Ba = (spa - sma) * rcp(spa + sma + eps);
    T Bb = (spb - smb) * rcp(spb + smb + eps);
    T r = T(2) * rcp(hsum);             // 1/hbar
    T cross = T(0.125) * (ua * Ba + ub * Bb);  // 1/4 (Ubar) x 1/2 (B)
    return (fabs(U) - U * U * r) * A - U * cross * r;
}

// One tile (index `tile`, row-major with ntx tiles per row) marched through
// all z planes by the whole CTA.
template <typename T, int TX, int TY, bool NONOSC>
__device__ __forceinline__ void single_tile(const Grid &g, T eps, int ntx, const T *__restrict__ h,
                                            const T *__restrict__ psi, const T *__restrict__ u1,
                                            const T *__restrict__ u2, const T *__restrict__ u3,
                                            T *__restrict__ out, int tile, T *const sm) {
    using L = Layout<TX, TY>;
    constexpr int EX = L::EX, PL = L::PL, NT = L::NT;
    const unsigned sm_base = (unsigned)__cvta_generic_to_shared(sm);
#define PLANE(k) (sm + (k) * PL)
#define RING(f, q) PLANE(L::RING + (f) * 4 + ((q) & 3))

    const int t = threadIdx.x;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int perx = g.per[0], pery = g.per[1], perz = g.per[2];
    const long long nxy = (long long)nx * ny;
    const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;

    // ---- this thread's column and its neighbour indices in the plane ----
    int rx, ry;
    onion<TX, TY>(t, rx, ry);
    const int gx = x0 + rx, gy = y0 + ry;
    const int c0 = (ry + 3) * EX + (rx + 3);
    // clamped cell neighbours (zero-gradient ghosts on lid axes)
    const int cL = c0 - ((!perx && gx == 0) ? 0 : 1);
    const int cR = c0 + ((!perx && gx == nx - 1) ? 0 : 1);
    const int cD = c0 - ((!pery && gy == 0) ? 0 : EX);
    const int cU = c0 + ((!pery && gy == ny - 1) ? 0 : EX);
    // lid faces of this column (zero velocity on its lower x / y face)
    const bool xlid = !perx && (gx <= 0 || gx >= nx);
    const bool ylid = !pery && (gy <= 0 || gy >= ny);
    const bool in_vm = t < L::N_VM, in_beta = t < L::N_BETA, in_v = t < L::N_V,
               in_out = t < L::N_OUT;
    const bool store = in_out && gx < nx && gy < ny;
    T *const outp = out + (long long)gy * nx + gx;

    // ---- load columns: row-major over the radius-3 plane ----
    int ld_cell[2], ld_u1[2], ld_u2[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        int c = t + r * NT;
        ld_cell[r] = ld_u1[r] = ld_u2[r] = -1;
        if (c < PL) {
            int lx = x0 - 3 + c % EX, ly = y0 - 3 + c / EX;
            int cx = wrap_or_clamp(lx, nx, perx), cy = wrap_or_clamp(ly, ny, pery);
            ld_cell[r] = cy * nx + cx;
            bool zx = !perx && (lx <= 0 || lx >= nx);  // lid x-face
            bool zy = !pery && (ly <= 0 || ly >= ny);  // lid y-face
            ld_u1[r] = zx ? -1 : ld_cell[r];
            ld_u2[r] = zy ? -1 : ld_cell[r];
        }
    }
    auto issue = [&](int p) {
        const long long pc = (long long)wrap_or_clamp(p, nz, perz) * nxy;
        const bool zz = !perz && (p <= 0 || p >= nz);  // lid z-face
        const unsigned slot = (unsigned)(p & 3) * PL;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int c = t + r * NT;
            if (c < PL) {
                const unsigned d = sm_base + (unsigned)(slot + c) * (unsigned)sizeof(T);
                const unsigned fs = 4u * PL * (unsigned)sizeof(T);  // field stride
                const long long o = pc + ld_cell[r];
                cp_async(d, psi + o, false);
                cp_async(d + fs, ld_u1[r] < 0 ? u1 : u1 + pc + ld_u1[r], ld_u1[r] < 0);
                cp_async(d + 2 * fs, ld_u2[r] < 0 ? u2 : u2 + pc + ld_u2[r], ld_u2[r] < 0);
                cp_async(d + 3 * fs, zz ? u3 : u3 + o, zz);
                cp_async(d + 4 * fs, h + o, false);
            }
        }
        cp_async_commit();
    };

    // ---- z range (periodic z also evaluates wrap planes around the ends) ----
    const int p_first = perz ? -3 : -1;
    const int p_last = nz + 2;
    const int q1lo = perz ? -2 : 0, q1hi = perz ? nz + 1 : nz - 1;
    const int q1top = perz ? q1hi : nz;                        // lid: plane nz is a ghost copy
    const int wlo = perz ? -2 : 0, whi = perz ? nz : nz - 2;   // z-face above plane q2
    const int vlo = perz ? -1 : 0, vhi = perz ? nz : nz - 1;   // V1, V2, beta at plane q2

    // ---- own-column queues along z ----
    T pn_mm = T(0), pn_m = T(0), pn_c = T(0);  // psi^n at q2-1, q2 (=q1-1), q1
    T p1a = T(0), p1b = T(0);                  // psi1 at q2-1, q2
    T sxa = T(0), sxb = T(0), sya = T(0), syb = T(0);  // pair sums at q2-1, q2
    T u1b = T(0), u2b = T(0), u3b = T(0), hb = T(1);   // inputs at q2
    T u3c = T(0);                              // u3 on the lower face of q1
    T wlo_v = T(0);                            // z-face pseudo-velocity below q2
    T bu_prev = T(0), bd_prev = T(0);          // limiter factors at q2-1
    T h_prev = T(1), p1_prev = T(0);           // h, psi1 at q3
    T dacc = T(0), gx_own = T(0), gy_own = T(0);

    issue(p_first);
    // FP32: unrolled by two so that the register queues shift by renaming
    // (FP64 would spill)
#pragma unroll(sizeof(T) == 4 ? 2 : 1)
    for (int p = p_first; p <= p_last; ++p) {
        const int q1 = p - 1, q2 = p - 2, q3 = p - 3;
        if (p + 1 <= p_last) issue(p + 1); else cp_async_commit();
        cp_async_wait_1();
        __syncthreads();  // (A) plane p landed; fluxes of the previous iteration visible

        // deferred: x/y part of the corrective divergence of plane q3
        if (in_out && q3 >= 0 && q3 <= nz - 1) {
            const T gxr = PLANE(L::GX)[c0 + 1], gyu = PLANE(L::GY)[c0 + EX];
            dacc = ((gxr - gx_own) + (gyu - gy_own)) + dacc;
        }

        // ---- (a1) donor-cell pass at plane q1 (all threads: radius 2) ----
        const T *Pn = RING(0, q1);
        const T pn_p = RING(0, p)[c0];
        const T u3p = RING(3, p)[c0];
        const T u1c = RING(1, q1)[c0], u2c = RING(2, q1)[c0], hc = RING(4, q1)[c0];
        T p1c = p1b;  // lid top ghost: zero-gradient copy of the plane below
        if (q1 >= q1lo && q1 <= q1hi) {
            const T fxl = upstream_flux(u1c, Pn[c0 - 1], pn_c);
            const T fxh = upstream_flux(RING(1, q1)[c0 + 1], pn_c, Pn[c0 + 1]);
            const T fyl = upstream_flux(u2c, Pn[c0 - EX], pn_c);
            const T fyh = upstream_flux(RING(2, q1)[c0 + EX], pn_c, Pn[c0 + EX]);
            const T fzl = upstream_flux(u3c, pn_m, pn_c);
            const T fzh = upstream_flux(u3p, pn_c, pn_p);
            const T div = (fxh - fxl) + (fyh - fyl) + (fzh - fzl);
            p1c = pn_c - div * rcp(hc);
        }
        if (q1 >= q1lo && q1 <= q1top) PLANE(L::P1 + (q1 & 1))[c0] = p1c;
        __syncthreads();  // (D) psi1 of plane q1 visible

        // ---- (a2) pseudo-velocities of the lower x/y faces at q2 ----
        const T *Pb = PLANE(L::P1 + (q2 & 1));
        const T *Pc = PLANE(L::P1 + (q1 & 1));
        T sxc = sxb, syc = syb;
        T v1_own = T(0), v2_own = T(0);
        T pl = T(0), pd = T(0);
        // pair sums across the lower x/y faces at q1 and across the z-face
        // between q2 and q1 (all threads: the cross terms read them one row
        // or column outside the pseudo-velocity region)
        if (q1 >= q1lo && q1 <= q1top) {
            sxc = Pc[c0 - 1] + p1c;
            syc = Pc[c0 - EX] + p1c;
            PLANE(L::SX + (q1 & 1))[c0] = sxc;
            PLANE(L::SY + (q1 & 1))[c0] = syc;
            PLANE(L::SZ)[c0] = p1b + p1c;
        }
        if (!perz && q1 == 0) { p1b = p1c; sxb = sxc; syb = syc; }  // lid bottom ghost
        if (in_v) {
            if (q2 >= vlo && q2 <= vhi) {
                const T *U1b = RING(1, q2), *U2b = RING(2, q2), *U3b = RING(3, q2),
                        *U3c = RING(3, q1), *Hb = RING(4, q2);
                const T *Sxb = PLANE(L::SX + (q2 & 1)), *Syb = PLANE(L::SY + (q2 & 1));
                pl = Pb[c0 - 1];
                pd = Pb[c0 - EX];
                // x-face: B_y from the x-pair sums of the rows above/below, B_z from own queue
                const T ua = U2b[c0 - 1] + u2b + U2b[c0 - 1 + EX] + U2b[c0 + EX];
                const T ub = U3b[c0 - 1] + u3b + U3c[c0 - 1] + u3c;
                const T v1 = pseudo_velocity(u1b, p1b, pl, Sxb[cU], Sxb[cD], ua, sxc, sxa, ub,
                                             Hb[c0 - 1] + hb, eps);
                // y-face: B_z from own queue, B_x from the y-pair sums of the columns left/right
                const T va = U3b[c0 - EX] + u3b + U3c[c0 - EX] + u3c;
                const T vb = U1b[c0 - EX] + u1b + U1b[c0 + 1 - EX] + U1b[c0 + 1];
                const T v2 = pseudo_velocity(u2b, p1b, pd, syc, sya, va, Syb[cR], Syb[cL], vb,
                                             Hb[c0 - EX] + hb, eps);
                v1_own = xlid ? T(0) : v1;
                v2_own = ylid ? T(0) : v2;
                PLANE(L::V1)[c0] = v1_own;
                PLANE(L::V2)[c0] = v2_own;
            }
        }
        __syncthreads();  // (F) V1, V2, pair sums of plane q2 visible

        // ---- (a2) z-face above q2, then (a3)+(a4) extrema and limiter factors ----
        T whi_v = T(0), bu_c = T(0), bd_c = T(0);
        if (in_beta) {
            if (q2 >= wlo && q2 <= whi) {
                const T *Sz = PLANE(L::SZ);
                const T *U1b = RING(1, q2), *U2b = RING(2, q2);
                const T ua = u1b + u1c + U1b[c0 + 1] + RING(1, q1)[c0 + 1];
                const T ub = u2b + u2c + U2b[c0 + EX] + RING(2, q1)[c0 + EX];
                whi_v = pseudo_velocity(u3c, p1c, p1b, Sz[cR], Sz[cL], ua, Sz[cU], Sz[cD], ub,
                                        hb + hc, eps);
            }
            if (NONOSC && q2 >= vlo && q2 <= vhi) {
                const T *Pnb = RING(0, q2);
                const T aL = Pnb[cL], aR = Pnb[cR], aD = Pnb[cD], aU = Pnb[cU];
                const T bL = Pb[cL], bR = Pb[cR], bD = Pb[cD], bU = Pb[cU];
                T mx = max3(max3(aL, aR, aD), max3(aU, bL, bR), max3(bD, bU, pn_mm));
                mx = max3(mx, max3(pn_m, pn_c, p1a), max3(p1b, p1c, p1b));
                T mn = min3(min3(aL, aR, aD), min3(aU, bL, bR), min3(bD, bU, pn_mm));
                mn = min3(mn, min3(pn_m, pn_c, p1a), min3(p1b, p1c, p1b));
                const T v1h = PLANE(L::V1)[c0 + 1], v2h = PLANE(L::V2)[c0 + EX];
                const T in = (pos(v1_own) * bL - neg(v1h) * bR) + (pos(v2_own) * bD - neg(v2h) * bU) +
                             (pos(wlo_v) * p1a - neg(whi_v) * p1c);
                const T outf = ((pos(v1h) - neg(v1_own)) + (pos(v2h) - neg(v2_own)) +
                                (pos(whi_v) - neg(wlo_v))) * p1b;
                bu_c = (mx - p1b) * hb * rcp(in + eps);
                bd_c = (p1b - mn) * hb * rcp(outf + eps);
                PLANE(L::BU)[c0] = bu_c;
                PLANE(L::BD)[c0] = bd_c;
            }
        }
        __syncthreads();  // (H) limiter factors of q2 visible; ring slot q2 free for reuse

        // ---- (a5)+(a6) limited corrective fluxes at q2, output of plane q3 ----
        if (in_vm && q2 >= 0 && q2 <= nz - 1) {
            T vm1 = v1_own, vm2 = v2_own;
            if (NONOSC) {
                const T *Bu = PLANE(L::BU), *Bd = PLANE(L::BD);
                const T buL = Bu[c0 - 1], bdL = Bd[c0 - 1], buD = Bu[c0 - EX], bdD = Bd[c0 - EX];
                vm1 = pos(v1_own) * min3(T(1), bdL, bu_c) + neg(v1_own) * min3(T(1), buL, bd_c);
                vm2 = pos(v2_own) * min3(T(1), bdD, bu_c) + neg(v2_own) * min3(T(1), buD, bd_c);
            }
            gx_own = xlid ? T(0) : upstream_flux(vm1, pl, p1b);
            gy_own = ylid ? T(0) : upstream_flux(vm2, pd, p1b);
            PLANE(L::GX)[c0] = gx_own;
            PLANE(L::GY)[c0] = gy_own;
        }
        const bool q3ok = q3 >= 0 && q3 <= nz - 1, q2ok = q2 >= 0 && q2 <= nz - 1;
        if (in_out && (q3ok || q2ok)) {
            // corrective flux through the z-face between q3 and q2 (zero on a lid)
            T gz = T(0);
            if (perz || (q2 >= 1 && q2 <= nz - 1)) {
                T vm3 = wlo_v;
                if (NONOSC)
                    vm3 = pos(wlo_v) * min3(T(1), bd_prev, bu_c) + neg(wlo_v) * min3(T(1), bu_prev, bd_c);
                gz = upstream_flux(vm3, p1a, p1b);
            }
            if (q3ok && store) outp[(long long)q3 * nxy] = p1_prev - (dacc + gz) * rcp(h_prev);
            dacc = -gz;  // lower z-face flux of plane q2; x/y parts are added next iteration
        }

        // ---- shift the queues ----
        h_prev = hb;
        p1_prev = p1b;
        pn_mm = pn_m;
        pn_m = pn_c;
        pn_c = pn_p;
        p1a = p1b;
        p1b = p1c;
        sxa = sxb;
        sxb = sxc;
        sya = syb;
        syb = syc;
        u1b = u1c;
        u2b = u2c;
        u3b = u3c;
        u3c = u3p;
        hb = hc;
        wlo_v = whi_v;
        bu_prev = bu_c;
        bd_prev = bd_c;
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();  // shared memory is reused by the next tile of a persistent CTA
#undef RING
#undef PLANE
}

template <typename T, int TX, int TY, bool NONOSC>
__global__ void __launch_bounds__(Layout<TX, TY>::NT, 1)
    k_fused(Grid g, T eps, int ntx, const T *__restrict__ h, const T *__restrict__ psi,
            const T *__restrict__ u1, const T *__restrict__ u2, const T *__restrict__ u3,
            T *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    single_tile<T, TX, TY, NONOSC>(g, eps, ntx, h, psi, u1, u2, u3, out, blockIdx.x,
                                   reinterpret_cast<T *>(smem_raw));
}

template <typename T, int TX, int TY>
cudaError_t launch_tile(const Grid &g, int nonosc, double eps, const void *h, const void *psi,
                        const void *u1, const void *u2, const void *u3, void *out,
                        cudaStream_t s) {
    using L = Layout<TX, TY>;
    const size_t smem = (size_t)L::NPLANES * L::PL * sizeof(T);
    const int ntx = (g.nx + TX - 1) / TX, nty = (g.ny + TY - 1) / TY;
    auto kern = nonosc ? k_fused<T, TX, TY, true> : k_fused<T, TX, TY, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ntx * nty, L::NT, smem, s>>>(g, (T)eps, ntx, (const T *)h, (const T *)psi,
                                        (const T *)u1, (const T *)u2, (const T *)u3, (T *)out);
    return cudaGetLastError();
}

}  // namespace

static bool single_tile_supported(int dtype, int tx, int ty) {
    if (dtype == MPDATA_F64) return (tx == 16 && ty == 16);
    return (tx == 32 && ty == 16) || (tx == 24 && ty == 24) || (tx == 16 && ty == 16) ||
           (tx == 24 && ty == 16);
}

bool fused_tile_supported(int dtype, const Grid &g, int tx, int ty) {
    if (dtype == MPDATA_F32 && fused_pairs_supported(g, tx, ty)) return true;
    return single_tile_supported(dtype, tx, ty);
}

void fused_default_tile(int dtype, const Grid &g, int nsm, int *tx, int *ty) {
    if (dtype == MPDATA_F64) { *tx = 16; *ty = 16; return; }
    // FP32: the tile of least predicted step time, waves x per-plane time of
    // a wave, waves = ceil(tiles / (SMs x CTAs per SM)).  Per-plane times
    // measured on GB300 (us, nz 33..63): a small grid (one wave) wants the
    // smallest, fastest plane; a large one the most cells per plane-time.
    // A tile of two CTAs per SM runs alone on its SM while the tiles do not
    // outnumber the SMs (us_one), two to an SM beyond (us per wave).
    struct Cand { int tx, ty, per_sm; double us_aligned, us_any, us_one_aligned, us_one_any; };
    static const Cand cands[] = {
        // two-column kernel; with nx % 4 == 0 (16-byte loads) the 32x12, 32x24
        // and 32x28 tiles add loader warps to their compute warps.  Medians
        // over serving-size grids: step time / (nz + 6)
        {32, 28, 1, 1.91, 2.38, 1.91, 2.38},
        {32, 24, 1, 1.67, 1.91, 1.67, 1.91},
        {32, 16, 1, 1.39, 1.45, 1.39, 1.45},
        {32, 12, 2, 1.78, 2.25, 1.11, 1.76},  // 9 compute warps + 1 loader warp, two CTAs per SM
        {24, 16, 1, 1.76, 1.76, 1.76, 1.76},  // one-column kernel
        {16, 16, 1, 1.44, 1.45, 1.44, 1.45},
    };
    const int sms = nsm > 0 ? nsm : 1 << 28;  // unknown device: every grid is one wave
    const bool a16 = g.nx % 4 == 0;
    double best = 0.0;
    for (const Cand &c : cands) {
        const long long tiles = (long long)((g.nx + c.tx - 1) / c.tx) * ((g.ny + c.ty - 1) / c.ty);
        const long long slots = (long long)sms * c.per_sm;
        const double t = tiles <= sms ? (a16 ? c.us_one_aligned : c.us_one_any)
                                      : (double)((tiles + slots - 1) / slots) * (a16 ? c.us_aligned : c.us_any);
        if (best == 0.0 || t < best * 0.98) { best = t; *tx = c.tx; *ty = c.ty; }
    }
}

namespace {

// Finish time of nA tiles of cost tA and then nB of cost tB handed out, each
// to the SM that frees first (the hardware starts the first launch's CTAs
// first).  SM loads take few distinct values, so they are kept as levels.
double handout_time(long long nA, double tA, long long nB, double tB, int nsm) {
    std::map<double, long long> lv;
    lv[0.0] = nsm;
    auto assign = [&](long long n, double t) {
        while (n > 0) {
            auto it = lv.begin();
            const double L = it->first;
            const long long c = it->second, k = std::min(c, n);
            if (k == c) lv.erase(it);
            else it->second -= k;
            lv[L + t] += k;
            n -= k;
        }
    };
    assign(nA, tA);
    assign(nB, tB);
    return lv.rbegin()->first;
}

}  // namespace

bool fused_band_plan(const Grid &g, int nsm, BandPlan *plan) {
    // Rows in 28-row bands of 32x28 tiles and 24-row bands of 32x24 tiles
    // (both with loader warps), run concurrently: SMs that finish early take the
    // next tile of either height, and the 24-row bands can end near ny where
    // one tile height would leave a mostly empty band.  Per-plane times as in
    // fused_default_tile; 0.02 x the 28-row plane time covers the fork and the
    // join.
    const double t28 = 1.91, t24 = 1.67;
    if (nsm <= 0 || g.nx % 4 != 0) return false;
    const long long ntx = (g.nx + 31) / 32;
    const long long w24 = (ntx * ((g.ny + 23) / 24) + nsm - 1) / nsm, w28 = (ntx * ((g.ny + 27) / 28) + nsm - 1) / nsm;
    const double single = std::min(w24 * t24, w28 * t28);
    // beyond 48 waves the last one is under 2 % of the step: not worth planning
    if (std::min(w24, w28) > 48) return false;
    double best = 0.0;
    for (int n28 = 1; 28 * n28 < g.ny; ++n28) {
        const int n24 = (g.ny - 28 * n28 + 23) / 24;
        const double t = handout_time(ntx * n28, t28, ntx * n24, t24, nsm) + 0.02 * t28;
        if (best == 0.0 || t < best) {
            best = t;
            plan->n28 = n28;
            plan->n24 = n24;
        }
    }
    return best > 0.0 && best < 0.99 * single;
}

cudaError_t launch_fused_step(int dtype, const Grid &g, int nonosc, double eps, int tx, int ty,
                              const void *h, const void *psi, const void *u1, const void *u2,
                              const void *u3, void *out, cudaStream_t s) {
    if (dtype == MPDATA_F32 && fused_pairs_supported(g, tx, ty))
        return launch_fused_pairs(g, nonosc, eps, tx, ty, h, psi, u1, u2, u3, out, s);
    if (dtype == MPDATA_F64) {
        if (tx == 16 && ty == 16)
            return launch_tile<double, 16, 16>(g, nonosc, eps, h, psi, u1, u2, u3, out, s);
        return cudaErrorInvalidValue;
    }
    if (tx == 32 && ty == 16)
        return launch_tile<float, 32, 16>(g, nonosc, eps, h, psi, u1, u2, u3, out, s);
    if (tx == 24 && ty == 24)
        return launch_tile<float, 24, 24>(g, nonosc, eps, h, psi, u1, u2, u3, out, s);
    if (tx == 24 && ty == 16)
        return launch_tile<float, 24, 16>(g, nonosc, eps, h, psi, u1, u2, u3, out, s);
    if (tx == 16 && ty == 16)
        return launch_tile<float, 16, 16>(g, nonosc, eps, h, psi, u1, u2, u3, out, s);
    return cudaErrorInvalidValue;
}

}  // namespace mpdata
