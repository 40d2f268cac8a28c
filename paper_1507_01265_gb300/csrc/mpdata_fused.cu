// Fused MPDATA step: every stage of one time step in one kernel (§5.2's
// 17 dependent stencil stages; the paper's (3+1)D decomposition in §5.3 keeps
// the intermediates of a block in cache -- here they live in shared memory
// and registers, so a step moves only the 5 input fields and the output
// through HBM).
//
// Decomposition (GB300-first, not the Xeon Phi code):
//   * a CTA owns an output tile of TX x TY columns and marches it through all
//     z planes; the z-neighbours of every quantity stay in registers as a
//     short queue, the x/y neighbours go through shared-memory planes;
//   * each stage is evaluated on exactly the columns later stages need
//     (psi1 on radius 2, pseudo-velocities on radius ~1.5, limiter factors
//     on radius 1, limited fluxes on radius 0..1); thread t owns one column,
//     columns are numbered from the tile outwards ring by ring, so every
//     stage's region is a prefix of the thread index and idle threads form
//     whole idle warps;
//   * inputs (psi, u1, u2, u3, h) of radius 3 stream into a 4-plane
//     shared-memory ring with cp.async one plane ahead of use; the zero-fill
//     form of cp.async supplies the zero velocity of lid faces;
//   * per plane: donor pass (plane p-1) -> pseudo-velocities (plane p-2 and
//     the z-face above it) -> limiter factors (p-2) -> limited fluxes and the
//     finished output (plane p-3).
//
// Boundary rules (the same readings as the oracle): periodic axes wrap; on a
// lid axis faces 0 and n carry zero velocity and ghost cells are
// zero-gradient copies (clamped neighbour reads in x/y, copied queue entries
// in z).
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
    static constexpr int NPLANES = 5 * 4 + 8;  // input ring + psi1 x2, v1, v2, bup, bdn, gx, gy
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
__device__ __forceinline__ void cp_async(T *dst, const T *src, bool zero) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    int bytes = zero ? 0 : (int)sizeof(T);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src),
                 "n"(sizeof(T)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <typename T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }

// Pseudo-velocity from its pieces:
//   V = (|U| - U^2/hbar) A - U (Ubar_a B_a + Ubar_b B_b) / hbar
template <typename T>
__device__ __forceinline__ T pseudo_velocity(T U, T pR, T pL, T spa, T sma, T ua, T spb, T smb,
                                             T ub, T h2sum, T eps) {
    T A = (pR - pL) / (pR + pL + eps);
    T Ba = T(0.5) * (spa - sma) / (spa + sma + eps);
    T Bb = T(0.5) * (spb - smb) / (spb + smb + eps);
    T hbar = T(0.5) * h2sum;
    return (fabs(U) - U * U / hbar) * A - U * (T(0.25) * ua * Ba + T(0.25) * ub * Bb) / hbar;
}

template <typename T, int TX, int TY, bool NONOSC>
__global__ void __launch_bounds__(Layout<TX, TY>::NT, 1)
    k_fused(Grid g, T eps, int ntx, const T *__restrict__ h, const T *__restrict__ psi,
            const T *__restrict__ u1, const T *__restrict__ u2, const T *__restrict__ u3,
            T *__restrict__ out) {
    using L = Layout<TX, TY>;
    constexpr int EX = L::EX, PL = L::PL, NT = L::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const sm = reinterpret_cast<T *>(smem_raw);
    // plane buffers
    T *const sV1 = sm + 22 * PL;
    T *const sV2 = sm + 23 * PL;
    T *const sBU = sm + 24 * PL;
    T *const sBD = sm + 25 * PL;
    T *const sGX = sm + 26 * PL;
    T *const sGY = sm + 27 * PL;
#define RING(f, q) (sm + ((f) * 4 + ((q) & 3)) * PL)
#define P1(q) (sm + (20 + ((q) & 1)) * PL)

    const int t = threadIdx.x;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int perx = g.per[0], pery = g.per[1], perz = g.per[2];
    const long long nxy = (long long)nx * ny;
    const int x0 = (blockIdx.x % ntx) * TX, y0 = (blockIdx.x / ntx) * TY;

    // ---- this thread's column and its neighbour indices in the plane ----
    int rx, ry;
    onion<TX, TY>(t, rx, ry);
    const int gx = x0 + rx, gy = y0 + ry;
    const int ex = rx + 3, ey = ry + 3;
    const int c0 = ey * EX + ex;
    int exL = ex - 1, exR = ex + 1, eyD = ey - 1, eyU = ey + 1;  // clamped cell neighbours
    if (!perx) { if (gx == 0) exL = ex; if (gx == nx - 1) exR = ex; }
    if (!pery) { if (gy == 0) eyD = ey; if (gy == ny - 1) eyU = ey; }
    const int cL = ey * EX + exL, cR = ey * EX + exR, cD = eyD * EX + ex, cU = eyU * EX + ex;
    // lid faces of this column (zero velocity on its lower x / y face)
    const bool xlid = !perx && (gx <= 0 || gx >= nx);
    const bool ylid = !pery && (gy <= 0 || gy >= ny);
    const bool in_vm = t < L::N_VM, in_beta = t < L::N_BETA, in_v = t < L::N_V,
               in_out = t < L::N_OUT;
    const bool store = in_out && gx < nx && gy < ny;

    // ---- load columns: row-major over the radius-3 plane ----
    int ld_cell[2], ld_u1[2], ld_u2[2];
    int nld = 0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        int c = t + r * NT;
        ld_cell[r] = ld_u1[r] = ld_u2[r] = -1;
        if (c < PL) {
            ++nld;
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
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (r < nld) {
                int c = t + r * NT;
                const long long o = pc + ld_cell[r];
                cp_async(RING(0, p) + c, psi + o, false);
                cp_async(RING(1, p) + c, ld_u1[r] < 0 ? u1 : u1 + pc + ld_u1[r], ld_u1[r] < 0);
                cp_async(RING(2, p) + c, ld_u2[r] < 0 ? u2 : u2 + pc + ld_u2[r], ld_u2[r] < 0);
                cp_async(RING(3, p) + c, zz ? u3 : u3 + o, zz);
                cp_async(RING(4, p) + c, h + o, false);
            }
        }
        cp_async_commit();
    };

    // ---- z range (periodic z also evaluates the wrap planes around the ends) ----
    const int p_first = perz ? -3 : -1;
    const int p_last = nz + 2;
    const int q1lo = perz ? -2 : 0, q1hi = perz ? nz + 1 : nz - 1;
    const int wlo = perz ? -2 : 0, whi = perz ? nz : nz - 2;   // z-face above plane q2
    const int vlo = perz ? -1 : 0, vhi = perz ? nz : nz - 1;   // V1, V2, beta at plane q2

    // ---- register queues along z ----
    T p1a = T(0), p1b = T(0);        // psi1 at q2-1, q2
    T sxa = T(0), sxb = T(0);        // x-pair sums at q2-1, q2
    T sya = T(0), syb = T(0);        // y-pair sums
    T wlo_v = T(0);                  // pseudo-velocity on the z-face below q2
    T bu_prev = T(0), bd_prev = T(0);// limiter factors at q2-1
    T pn_prev = T(0);                // psi^n at q2-1
    T h_prev = T(1);                 // h at q3
    T dacc = T(0);                   // partial divergence of the output plane
    T gx_own = T(0), gy_own = T(0);  // own lower-face corrective fluxes (previous plane)
    T v1_own = T(0), v2_own = T(0);

    issue(p_first);
    for (int p = p_first; p <= p_last; ++p) {
        const int q1 = p - 1, q2 = p - 2, q3 = p - 3;
        if (p + 1 <= p_last) issue(p + 1); else cp_async_commit();
        cp_async_wait_1();
        __syncthreads();  // (A) plane p landed; previous iteration's fluxes visible

        // deferred: finish the x/y divergence of plane q3 (fluxes of the previous iteration)
        if (in_out && q3 >= 0 && q3 <= nz - 1) {
            T gxr = sGX[c0 + 1], gyu = sGY[c0 + EX];
            dacc = ((gxr - gx_own) + (gyu - gy_own)) + dacc;
        }

        // (a1) donor-cell pass at plane q1
        T p1c = p1b;  // lid top ghost: zero-gradient copy
        if (q1 >= q1lo && q1 <= q1hi) {
            const T *pm = RING(0, q1 - 1), *pc = RING(0, q1), *pp = RING(0, q1 + 1);
            const T *U1 = RING(1, q1), *U2 = RING(2, q1), *U3c = RING(3, q1),
                    *U3p = RING(3, q1 + 1);
            T ps = pc[c0];
            T fxl = upstream_flux(U1[c0], pc[c0 - 1], ps);
            T fxh = upstream_flux(U1[c0 + 1], ps, pc[c0 + 1]);
            T fyl = upstream_flux(U2[c0], pc[c0 - EX], ps);
            T fyh = upstream_flux(U2[c0 + EX], ps, pc[c0 + EX]);
            T fzl = upstream_flux(U3c[c0], pm[c0], ps);
            T fzh = upstream_flux(U3p[c0], ps, pp[c0]);
            T div = (fxh - fxl) + (fyh - fyl) + (fzh - fzl);
            p1c = ps - div / RING(4, q1)[c0];
        }
        if (q1 >= q1lo && q1 <= (perz ? q1hi : nz)) P1(q1)[c0] = p1c;
        __syncthreads();  // (D) psi1 plane q1 visible

        // own h and psi^n at q2, read now: after the last barrier of this
        // iteration other threads may already stream plane p+2 into this slot
        const T h_q2 = RING(4, q2)[c0], pn_q2 = RING(0, q2)[c0];

        // (a2) pseudo-velocities: lower x/y faces at q2, z-face between q2 and q1
        T sxc = sxb, syc = syb, whi_v = T(0);
        if (in_v) {
            const T *Pb = P1(q2), *Pc = P1(q1);
            const bool q1ok = q1 >= q1lo && q1 <= (perz ? q1hi : nz);
            if (q1ok) {
                sxc = Pc[c0 - 1] + p1c;
                syc = Pc[c0 - EX] + p1c;
            }
            if (!perz && q1 == 0) { p1b = p1c; sxb = sxc; syb = syc; }  // lid bottom ghost
            if (q2 >= vlo && q2 <= vhi) {
                const T *U1b = RING(1, q2), *U2b = RING(2, q2), *U3b = RING(3, q2),
                        *U3c = RING(3, q1), *Hb = RING(4, q2);
                const T pb = p1b;
                // x-face
                {
                    T U = U1b[c0];
                    T pl = Pb[c0 - 1];
                    T spa = Pb[cU] + Pb[cU - 1], sma = Pb[cD] + Pb[cD - 1];
                    T ua = U2b[c0 - 1] + U2b[c0] + U2b[c0 - 1 + EX] + U2b[c0 + EX];
                    T ub = U3b[c0 - 1] + U3b[c0] + U3c[c0 - 1] + U3c[c0];
                    T v = pseudo_velocity(U, pb, pl, spa, sma, ua, sxc, sxa, ub,
                                          Hb[c0 - 1] + Hb[c0], eps);
                    v1_own = xlid ? T(0) : v;
                }
                // y-face
                {
                    T U = U2b[c0];
                    T pd = Pb[c0 - EX];
                    T ua = U3b[c0 - EX] + U3b[c0] + U3c[c0 - EX] + U3c[c0];
                    T spb = Pb[cR] + Pb[cR - EX], smb = Pb[cL] + Pb[cL - EX];
                    T ub = U1b[c0 - EX] + U1b[c0] + U1b[c0 + 1 - EX] + U1b[c0 + 1];
                    T v = pseudo_velocity(U, pb, pd, syc, sya, ua, spb, smb, ub,
                                          Hb[c0 - EX] + Hb[c0], eps);
                    v2_own = ylid ? T(0) : v;
                }
                sV1[c0] = v1_own;
                sV2[c0] = v2_own;
            }
            if (q2 >= wlo && q2 <= whi) {
                const T *U1b = RING(1, q2), *U2b = RING(2, q2), *U1c = RING(1, q1),
                        *U2c = RING(2, q1);
                T U = RING(3, q1)[c0];
                T spa = Pc[cR] + Pb[cR], sma = Pc[cL] + Pb[cL];
                T ua = U1b[c0] + U1c[c0] + U1b[c0 + 1] + U1c[c0 + 1];
                T spb = Pc[cU] + Pb[cU], smb = Pc[cD] + Pb[cD];
                T ub = U2b[c0] + U2c[c0] + U2b[c0 + EX] + U2c[c0 + EX];
                whi_v = pseudo_velocity(U, p1c, p1b, spa, sma, ua, spb, smb, ub,
                                        RING(4, q2)[c0] + RING(4, q1)[c0], eps);
            }
        }
        __syncthreads();  // (F) V1, V2 of plane q2 visible

        // (a3)+(a4) local extrema and limiter factors at q2
        T bu_c = T(0), bd_c = T(0);
        if (NONOSC) {
            if (in_beta && q2 >= vlo && q2 <= vhi) {
                const T *Pn = RING(0, q2), *Pb = P1(q2);
                T pnc = Pn[c0], pnu = RING(0, q1)[c0];
                T mx = tmax(tmax(pnc, p1b), tmax(pn_prev, pnu));
                T mn = tmin(tmin(pnc, p1b), tmin(pn_prev, pnu));
                mx = tmax(mx, tmax(p1a, p1c));
                mn = tmin(mn, tmin(p1a, p1c));
                T aL = Pn[cL], aR = Pn[cR], aD = Pn[cD], aU = Pn[cU];
                T bL = Pb[cL], bR = Pb[cR], bD = Pb[cD], bU = Pb[cU];
                mx = tmax(mx, tmax(tmax(aL, aR), tmax(aD, aU)));
                mx = tmax(mx, tmax(tmax(bL, bR), tmax(bD, bU)));
                mn = tmin(mn, tmin(tmin(aL, aR), tmin(aD, aU)));
                mn = tmin(mn, tmin(tmin(bL, bR), tmin(bD, bU)));
                T v1h = sV1[c0 + 1], v2h = sV2[c0 + EX];
                T in = (tmax(v1_own, T(0)) * bL - tmin(v1h, T(0)) * bR) +
                       (tmax(v2_own, T(0)) * bD - tmin(v2h, T(0)) * bU) +
                       (tmax(wlo_v, T(0)) * p1a - tmin(whi_v, T(0)) * p1c);
                T outf = ((tmax(v1h, T(0)) - tmin(v1_own, T(0))) +
                          (tmax(v2h, T(0)) - tmin(v2_own, T(0))) +
                          (tmax(whi_v, T(0)) - tmin(wlo_v, T(0)))) * p1b;
                T hc = RING(4, q2)[c0];
                bu_c = (mx - p1b) * hc / (in + eps);
                bd_c = (p1b - mn) * hc / (outf + eps);
                sBU[c0] = bu_c;
                sBD[c0] = bd_c;
            }
            __syncthreads();  // (H) limiter factors of plane q2 visible
        }

        // (a5)+(a6) limited velocities, corrective fluxes, and the output of plane q3
        if (in_vm && q2 >= 0 && q2 <= nz - 1) {
            const T *Pb = P1(q2);
            T vm1 = v1_own, vm2 = v2_own;
            if (NONOSC) {
                T buL = sBU[c0 - 1], bdL = sBD[c0 - 1], buD = sBU[c0 - EX], bdD = sBD[c0 - EX];
                vm1 = tmax(v1_own, T(0)) * tmin(T(1), tmin(bdL, bu_c)) +
                      tmin(v1_own, T(0)) * tmin(T(1), tmin(buL, bd_c));
                vm2 = tmax(v2_own, T(0)) * tmin(T(1), tmin(bdD, bu_c)) +
                      tmin(v2_own, T(0)) * tmin(T(1), tmin(buD, bd_c));
            }
            gx_own = xlid ? T(0) : upstream_flux(vm1, Pb[c0 - 1], p1b);
            gy_own = ylid ? T(0) : upstream_flux(vm2, Pb[c0 - EX], p1b);
            sGX[c0] = gx_own;
            sGY[c0] = gy_own;
        }
        const bool q3ok = q3 >= 0 && q3 <= nz - 1, q2ok = q2 >= 0 && q2 <= nz - 1;
        if (in_out && (q3ok || q2ok)) {
            // corrective flux through the z-face between q3 and q2 (zero on a lid)
            T gz = T(0);
            if (perz || (q2 >= 1 && q2 <= nz - 1)) {
                T vm3 = wlo_v;
                if (NONOSC)
                    vm3 = tmax(wlo_v, T(0)) * tmin(T(1), tmin(bd_prev, bu_c)) +
                          tmin(wlo_v, T(0)) * tmin(T(1), tmin(bu_prev, bd_c));
                gz = upstream_flux(vm3, p1a, p1b);
            }
            if (q3ok) {
                T res = p1a - (dacc + gz) / h_prev;
                if (store) out[(long long)q3 * nxy + (long long)gy * nx + gx] = res;
            }
            dacc = -gz;  // lower z-face flux of plane q2; x/y parts are added next iteration
        }

        // shift the queues
        h_prev = h_q2;
        pn_prev = pn_q2;
        p1a = p1b;
        p1b = p1c;
        sxa = sxb;
        sxb = sxc;
        sya = syb;
        syb = syc;
        wlo_v = whi_v;
        bu_prev = bu_c;
        bd_prev = bd_c;
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
#undef RING
#undef P1
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

bool fused_tile_supported(int dtype, int tx, int ty) {
    if (dtype == MPDATA_F64) return (tx == 16 && ty == 16);
    return (tx == 32 && ty == 16) || (tx == 24 && ty == 24) || (tx == 16 && ty == 16);
}

void fused_default_tile(int dtype, int *tx, int *ty) {
    if (dtype == MPDATA_F64) { *tx = 16; *ty = 16; }
    else { *tx = 32; *ty = 16; }
}

cudaError_t launch_fused_step(int dtype, const Grid &g, int nonosc, double eps, int tx, int ty,
                              const void *h, const void *psi, const void *u1, const void *u2,
                              const void *u3, void *out, cudaStream_t s) {
    if (dtype == MPDATA_F64) {
        if (tx == 16 && ty == 16)
            return launch_tile<double, 16, 16>(g, nonosc, eps, h, psi, u1, u2, u3, out, s);
        return cudaErrorInvalidValue;
    }
    if (tx == 32 && ty == 16)
        return launch_tile<float, 32, 16>(g, nonosc, eps, h, psi, u1, u2, u3, out, s);
    if (tx == 24 && ty == 24)
        return launch_tile<float, 24, 24>(g, nonosc, eps, h, psi, u1, u2, u3, out, s);
    if (tx == 16 && ty == 16)
        return launch_tile<float, 16, 16>(g, nonosc, eps, h, psi, u1, u2, u3, out, s);
    return cudaErrorInvalidValue;
}

}  // namespace mpdata
