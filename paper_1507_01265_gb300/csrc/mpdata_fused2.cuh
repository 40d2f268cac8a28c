// Fused MPDATA step, FP32, two adjacent x-columns per thread.
//
// A CTA marches a TX x TY tile through z (TX = 32; TY = 12, 16, 24 or 28).  Per
// iteration p, with q1 = p-1, q2 = p-2, q3 = p-3, three barriers:
//   alpha  donor pass of q1 completed from the neighbours' fluxes (a1), pair
//          sums for the cross terms, x/y pseudo-velocities at q2 (a2);
//   beta   z-face pseudo-velocity, local extrema and limiter factors at q2
//          (a2-a4);
//   gamma  limited velocities and corrective fluxes at q2, output of q3
//          (a5-a6), and the donor fluxes of plane p (work for the warps that
//          the flux stage leaves idle).
// Inputs (psi, u1, u2, u3, h) load two planes ahead into a 4-plane ring.
// Aimed at the instruction count and latency, which bound this step on GB300:
//   * each thread owns a pair of adjacent columns (i, i+1) and evaluates both
//     with packed f32x2 add/mul/fma, so per-thread overhead (addressing,
//     predicates, loop control) is paid once per two cells and shared-memory
//     neighbours of the pair come in one 64-bit load; the interior planes
//     run in blocks of four so that ring slots are compile-time constants and
//     register queues shift by renaming;
//   * inputs stream in as 16-byte cp.async chunks when nx is a multiple of 4
//     (chunks then never straddle a wrap or a lid and rows stay 16-byte
//     aligned); for any other nx as 4-byte copies in element order (a warp
//     copies 128 contiguous bytes).  Columns past nx are ghosts: wrapped
//     copies on a periodic axis, zero-filled faces and clamped cell values
//     behind a lid, never stored;
//   * when x and y are both periodic (LID = false) every neighbour offset is
//     a compile-time constant; with a lid on x or y (LID = true) the neighbour
//     reads of cell fields are clamped (zero-gradient ghosts) and the lid
//     faces are forced to zero velocity.
// Threads are numbered from the tile outwards ring by ring in pair units, so
// each stage's region is a prefix of the thread index.
// The 32x24 and 32x28 tiles of a grid with nx % 4 == 0 add two loader warps
// to their 16 / 18 compute warps, the 32x12 tile one to its 9 (pairs_loader):
// they issue and wait for every input load, so the compute threads hold no
// load state (fewer spills) and no load instructions.  The 32x12 tile's
// 104 KB of shared memory let two CTAs share an SM, so that one CTA's warps
// run while the other's wait at a barrier.
#pragma once

#include <type_traits>

#include "mpdata_internal.cuh"

namespace mpdata {

// One launch of the two-column kernel over tile rows [y0, y0 + TY * nty).
struct PairsRows {
    Grid g;
    int nonosc;
    double eps;
    int y0, nty;
    const void *h, *psi, *u1, *u2, *u3;
    void *out;
    cudaStream_t s;
};

namespace {

using F2 = float2;

__device__ __forceinline__ F2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ F2 add(F2 a, F2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ F2 mul(F2 a, F2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ F2 sub(F2 a, F2 b) {
    unsigned long long ra, rb, rc;
    asm("mov.b64 %0, {%1,%2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1,%2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rc) : "l"(ra), "l"(rb));
    F2 r;
    asm("mov.b64 {%0,%1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(rc));
    return r;
}
__device__ __forceinline__ float rcp1(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ F2 rcp(F2 a) { return make_float2(rcp1(a.x), rcp1(a.y)); }
__device__ __forceinline__ F2 fabs2(F2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ F2 pos(F2 a) { return make_float2(fmaxf(a.x, 0.f), fmaxf(a.y, 0.f)); }
__device__ __forceinline__ F2 neg(F2 a) { return make_float2(fminf(a.x, 0.f), fminf(a.y, 0.f)); }
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ F2 max3(F2 a, F2 b, F2 c) {
    return make_float2(max3f(a.x, b.x, c.x), max3f(a.y, b.y, c.y));
}
__device__ __forceinline__ F2 min3(F2 a, F2 b, F2 c) {
    return make_float2(min3f(a.x, b.x, c.x), min3f(a.y, b.y, c.y));
}
// Upstream flux [U]+ L + [U]- R of each column of the pair.
__device__ __forceinline__ F2 flux(F2 U, F2 L, F2 R) {
    return mul(U, make_float2(U.x > 0.f ? L.x : R.x, U.y > 0.f ? L.y : R.y));
}
__device__ __forceinline__ void st2(float *p, F2 v) { *reinterpret_cast<F2 *>(p) = v; }

// Pseudo-velocity of both faces of the pair (see mpdata_fused.cu):
//   V = (|U| - U^2/hbar) A - U (Ubar_a B_a + Ubar_b B_b) / hbar
__device__ __forceinline__ F2 pseudo_velocity(F2 U, F2 pR, F2 pL, F2 psum, F2 spa, F2 sma, F2 ua,
                                              F2 spb, F2 smb, F2 ub, F2 hsum, F2 eps) {
    const F2 A = mul(sub(pR, pL), rcp(add(psum, eps)));
    const F2 Ba = mul(sub(spa, sma), rcp(add(add(spa, sma), eps)));
    const F2 Bb = mul(sub(spb, smb), rcp(add(add(spb, smb), eps)));
    // t = U / hbar = 2U / hsum; the 1/4 (Ubar) x 1/2 (B) of the cross term
    // rides on t/8.  The power-of-two scalings are exact, so this is the
    // same value as scaling after the reciprocal, one step shorter.
    const F2 rh = rcp(hsum);
    const F2 t = mul(add(U, U), rh);
    const F2 t8 = mul(mul(bc(0.25f), U), rh);
    return sub(mul(sub(fabs2(U), mul(U, t)), A), mul(t8, fma2(ua, Ba, mul(ub, Bb))));
}

// Shared-memory planes: rows of EXL = TX + 8 loaded columns at a pitch of
// EX = EXL + 4 words.  The halo threads of the onion order include two
// vertical strips (one column pair, consecutive rows in consecutive lanes);
// with a pitch of 40 words (8 mod 32) a strip's 32 lanes fall on 4 bank
// positions, with 44 (12 mod 32) on 8, which halves the wavefronts of every
// strip access.  The pitch stays a multiple of 4 words so that rows stay
// 16-byte aligned for the 16-byte cp.async (a pitch of 42 would spread the
// strips over 16 positions but needs 8-byte copies, which go through L1 and
// evict the kernel's spill lines).
template <int TX, int TY, int NR_ = 5>
struct Lay2 {
    static constexpr int NLD = TY == 12 ? 32 : 64;  // loader threads (with loader warps)
    static constexpr int MINB = TY == 12 ? 2 : 1;   // CTAs per SM
    static_assert(TX % 4 == 0, "TX must be a multiple of 4");
    static constexpr int HX = TX / 2;           // output pairs per row
    static constexpr int NPX = HX + 2;          // pairs of the radius-2 regions
    static constexpr int EXL = TX + 8;          // loaded plane row: columns -4 .. TX+3
    static constexpr int EX = EXL + 4;          // row pitch (words)
    static constexpr int EY = TY + 6;           // plane rows: -3 .. TY+2
    static constexpr int PL = EX * EY;
    static constexpr int PLL = EXL * EY;        // loaded elements per plane
    static constexpr int NT = NPX * (TY + 4);   // psi1 region = threads
    static constexpr int NTW = (NT + 31) / 32 * 32;  // NT in whole warps
    static constexpr int N_OUT = HX * TY;
    static constexpr int N_VM = (HX + 1) * (TY + 1);
    static constexpr int N_BETA = NPX * (TY + 2);
    static constexpr int N_V = NPX * (TY + 3);
    static constexpr int CPR = EXL / 4;         // 16-byte chunks per plane row
    static constexpr int NCH = CPR * EY;
    static_assert(NCH <= NT, "one load chunk per thread");
    static constexpr int NR = NR_;              // input ring depth (planes)
    static constexpr int RING = 0, P1 = 5 * NR, SX = P1 + 2, SY = SX + 2, SZ = SY + 2;
    static constexpr int V1 = SZ + 1, V2 = V1 + 1, BU = V2 + 1, BD = BU + 1, GX = BD + 1, GY = GX + 1;
    static constexpr int NPLANES = GY + 1;
};

// Pair (px, row) of thread t; pair px covers columns 2px-4, 2px-3 of the tile.
// Rings outwards, each stage's region a prefix of t:
//   out (HX x TY) | N_VM: row TY, col-pair HX+2 rows [0,TY] |
//   N_BETA: col-pair 1 rows [-1,TY], row -1 | N_V: row TY+1 | NT: row -2.
// Within a ring the row comes before the strip in N_VM and after it in
// N_BETA, so that no warp holds more than 19 lanes of a vertical strip (whose
// lanes are one row pitch apart and share 8 bank positions).
template <int TX, int TY>
__device__ __forceinline__ void onion2(int t, int &px, int &ry) {
    using L = Lay2<TX, TY>;
    constexpr int HX = L::HX;
    if (t < L::N_OUT) { px = 2 + t % HX; ry = t / HX; return; }
    if (t >= L::NT) { px = HX + 4; ry = t - L::NT; return; }  // idle: row padding
    t -= L::N_OUT;
    if (t < HX) { px = 2 + t; ry = TY; return; }
    t -= HX;
    if (t < TY + 1) { px = HX + 2; ry = t; return; }
    t -= TY + 1;
    if (t < TY + 2) { px = 1; ry = t - 1; return; }
    t -= TY + 2;
    if (t < HX + 1) { px = 2 + t; ry = -1; return; }
    t -= HX + 1;
    if (t < HX + 2) { px = 1 + t; ry = TY + 1; return; }
    t -= HX + 2;
    px = 1 + t;
    ry = -2;
}

__device__ __forceinline__ int slot5(int q) {
    const int r = q % 5;
    return r < 0 ? r + 5 : r;
}

__device__ __forceinline__ int wrap(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

__device__ __forceinline__ void cp16(unsigned dst, const float *src, bool zero) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
                 "r"(zero ? 0 : 16)
                 : "memory");
}
__device__ __forceinline__ void cp4(unsigned dst, const float *src, bool zero) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src),
                 "r"(zero ? 0 : 4)
                 : "memory");
}

// Shared-memory access with explicit 32-bit addresses: one per-thread base
// plus per-iteration slot bases; every field, plane and neighbour offset is a
// compile-time immediate of the load/store.
template <int OFF>
__device__ __forceinline__ F2 ldp(unsigned b) {
    F2 v;
    asm volatile("ld.shared.v2.f32 {%0,%1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(b), "n"(OFF));
    return v;
}
template <int OFF>
__device__ __forceinline__ float lds(unsigned b) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(b), "n"(OFF));
    return v;
}
template <int OFF>
__device__ __forceinline__ void stp(unsigned b, F2 v) {
    asm volatile("st.shared.v2.f32 [%0+%1], {%2,%3};" ::"r"(b), "n"(OFF), "f"(v.x), "f"(v.y) : "memory");
}

// ---------------------------------------------------------------------------
// One tile (tile index `tile` of grid a.g, tiles numbered row-major with
// a.ntx tiles per row) marched through all z planes by the whole CTA.
// AL: 1 = nx % 4 == 0 (16-byte loads, 8-byte stores), 0 = any nx (4-byte
// loads, per-column stores), 2 = decided per tile from nx.
// Inputs sit in a 4-plane ring: plane p in slot (p - p_first) & 3, its loads
// issued after the second barrier of iteration p - 2, into the slot that
// plane p - 4 has just freed (it arrives within one iteration).  The interior
// iterations (3 <= p <= nz - 3: every stage active, every load inside the
// grid) run in blocks of four whose slot offsets are compile-time constants
// and which carry no z-range checks; the first and last few iterations run
// one body that checks the z range and computes the slots at run time.
template <int V>
using IC = std::integral_constant<int, V>;
using BT = std::integral_constant<bool, true>;
using BF = std::integral_constant<bool, false>;

// Loader warps of the two-column tile (k_fused_pairs with LD): threads NTW ..
// NTW + NLD - 1 issue every 16-byte input load of the tile and wait for them, on
// the same schedule and with the same barriers (three per plane and one at the
// end) as pairs_tile, so that the compute threads carry no load state.
template <int TX, int TY, bool LID>
__device__ __forceinline__ void pairs_loader(const TileArgs &a, int tile, float *sm) {
    using L = Lay2<TX, TY, 4>;
    constexpr int NLD = L::NLD;
    constexpr int KCH = (L::NCH + NLD - 1) / NLD;
    static_assert(KCH <= 8, "chunk flags are packed 8 per byte");
    constexpr int PL = L::PL, PB = PL * 4, FB = L::NR * PB, EX = L::EX;
    const Grid &g = a.g;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int perx = LID ? g.per[0] : 1, pery = LID ? g.per[1] : 1, perz = g.per[2];
    const long long nxy = (long long)nx * ny;
    const int ntx = a.ntx;
    const int x0 = (tile % ntx) * TX, y0 = a.y0 + (tile / ntx) * TY;
    const unsigned sm_base = (unsigned)__cvta_generic_to_shared(sm);
    const int j = threadIdx.x - L::NTW;
    int ld_off[KCH];
    unsigned ld_dst[KCH];
    unsigned cfl = 0;  // per chunk k: bit k has, 8+k lid ghost, 16+k y-lid face, 24+k x-lid face
#pragma unroll
    for (int k = 0; k < KCH; ++k) {
        const int c = j + k * NLD;
        ld_off[k] = 0;
        ld_dst[k] = 0;
        if (c < L::NCH) {
            const int ey = c / L::CPR, cc = c % L::CPR;
            const int lx = x0 - 4 + 4 * cc, ly = y0 - 3 + ey;
            int cx, cy;
            bool outx = false, outy = false;
            if (perx) cx = wrap(lx, nx); else { outx = lx < 0 || lx >= nx; cx = outx ? 0 : lx; }
            if (pery) cy = wrap(ly, ny); else { outy = ly < 0 || ly >= ny; cy = outy ? 0 : ly; }
            const bool za = outx || outy;
            cfl |= 1u << k;
            cfl |= (unsigned)za << (8 + k);
            cfl |= (unsigned)(za || (!pery && ly == 0)) << (16 + k);
            cfl |= (unsigned)(LID && !perx && lx == 0) << (24 + k);
            ld_off[k] = cy * nx + cx;
            ld_dst[k] = sm_base + (unsigned)(ey * EX + 4 * cc) * 4u;
        }
    }
    auto issue = [&](int p, unsigned so) {
        const long long pz = (long long)(perz ? wrap(p, nz) : min(max(p, 0), nz - 1));
        const bool zz = !perz && (p <= 0 || p >= nz);
#pragma unroll
        for (int k = 0; k < KCH; ++k) {
            if ((cfl >> k) & 1u) {
                const long long pc = pz * nxy + ld_off[k];
                const unsigned d = ld_dst[k] + so;
                const bool za = (cfl >> (8 + k)) & 1u, zu2 = (cfl >> (16 + k)) & 1u;
                cp16(d, a.psi + pc, za);
                cp16(d + FB, a.u1 + pc, za);
                cp16(d + 2 * FB, a.u2 + pc, zu2);
                cp16(d + 3 * FB, a.u3 + pc, za || zz);
                cp16(d + 4 * FB, a.h + pc, za);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    const int p_first = perz ? -3 : -1, p_last = nz + 2;
    issue(p_first, 0u);
    issue(p_first + 1, (unsigned)PB);
#pragma unroll 1
    for (int p = p_first; p <= p_last; ++p) {
        const int kk = (p - p_first) & 3;
        __syncthreads();  // (F)
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // plane p+1 landed
        if (LID) {
#pragma unroll
            for (int k = 0; k < KCH; ++k)
                if ((cfl >> (24 + k)) & 1u)
                    sm[(ld_dst[k] - sm_base) / 4u + (unsigned)(L::NR * PL + ((kk + 1) & 3) * PL)] = 0.f;
        }
        __syncthreads();  // (H)
        if (p + 2 <= p_last) issue(p + 2, (unsigned)(((kk + 2) & 3) * PB));
        __syncthreads();  // (X)
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
}

template <int TX, int TY, bool NONOSC, bool LID, int AL, bool LD = false>
__device__ __forceinline__ void pairs_tile(const TileArgs &a, int tile, float *sm) {
    using L = Lay2<TX, TY, 4>;
    static_assert(!LD || AL == 1, "loader warps take the 16-byte loads only");
    // __syncthreads is an aligned barrier: every warp must reach each one at
    // one code location, so the loader threads form whole warps and the
    // threads NT .. NTW - 1 that fill the last compute warp run the compute
    // path idle, placed by onion2 on the row padding (idle thread k stores to
    // words 2HX + 8, 2HX + 9 of row k + 3 of a plane and reads one word and
    // one row around them; no stage touches those words)
    static_assert(!LD || L::NTW - L::NT <= L::EY - 4, "idle threads: one padding row each");
    static_assert(!LD || 2 * (L::HX + 4) + 3 <= L::EX, "idle threads stay inside the row pitch");
    const Grid &g = a.g;
    const float eps1 = a.eps;
    const float *__restrict__ h = a.h;
    const float *__restrict__ psi = a.psi;
    const float *__restrict__ u1 = a.u1;
    const float *__restrict__ u2 = a.u2;
    const float *__restrict__ u3 = a.u3;
    float *__restrict__ out = a.out;
    const int ntx = a.ntx;
    constexpr int EX = L::EX, EXL = L::EXL, PL = L::PL, PLL = L::PLL;
    constexpr int PB = PL * 4;         // bytes per plane
    constexpr int FB = L::NR * PB;     // bytes between ring fields
    constexpr int RB = EX * 4;         // bytes per plane row
    constexpr int oP1 = L::P1 * PB, oSX = L::SX * PB, oSY = L::SY * PB, oSZ = L::SZ * PB;
    constexpr int oV1 = L::V1 * PB, oV2 = L::V2 * PB, oBU = L::BU * PB, oBD = L::BD * PB;
    constexpr int oGX = L::GX * PB, oGY = L::GY * PB;
    const unsigned sm_base = (unsigned)__cvta_generic_to_shared(sm);

    const int t = threadIdx.x;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int perx = LID ? g.per[0] : 1, pery = LID ? g.per[1] : 1, perz = g.per[2];
    const long long nxy = (long long)nx * ny;
    const int x0 = (tile % ntx) * TX, y0 = a.y0 + (tile / ntx) * TY;
    const F2 eps = bc(eps1);

    if constexpr (LD) {
        if (t >= L::NTW) {
            pairs_loader<TX, TY, LID>(a, tile, sm);
            return;
        }
    }
    int px, ry;
    onion2<TX, TY>(t, px, ry);
    const int gx = x0 + 2 * px - 4, gy = y0 + ry;
    const unsigned tb = sm_base + (unsigned)((ry + 3) * EX + 2 * px) * 4u;
    const bool clampL = LID && !perx && gx == 0;
    const bool clampR = LID && !perx && gx + 1 == nx - 1;
    const int dD = (LID && !pery && gy == 0) ? 0 : -RB;
    const int dU = (LID && !pery && gy == ny - 1) ? 0 : RB;
    const bool clampRx = LID && AL != 1 && !perx && gx == nx - 1;
    const bool a16 = AL == 1 || (AL == 2 && (nx & 3) == 0);
    const bool xlid0 = LID && !perx && (gx <= 0 || gx >= nx);
    const bool xlid1 = LID && !perx && (gx + 1 <= 0 || gx + 1 >= nx);
    const bool ylid = LID && !pery && (gy <= 0 || gy >= ny);
    const bool in_vm = t < L::N_VM, in_beta = t < L::N_BETA, in_v = t < L::N_V,
               in_out = t < L::N_OUT;
    const bool store = in_out && gx < nx && gy < ny;
    float *const outp = out + (long long)gy * nx + gx;

    auto ldD = [&](unsigned b) { if constexpr (LID) return ldp<0>(b + dD); else return ldp<-RB>(b); };
    auto ldU = [&](unsigned b) { if constexpr (LID) return ldp<0>(b + dU); else return ldp<RB>(b); };
    auto lshC = [&](unsigned b, F2 own) { float v = lds<-4>(b); return make_float2(clampL ? own.x : v, own.x); };
    auto rshC = [&](unsigned b, F2 own) {
        float v = lds<8>(b);
        return make_float2(clampRx ? own.x : own.y, clampR ? own.y : v);
    };
    auto lshF = [&](unsigned b, F2 own) { return make_float2(lds<-4>(b), own.x); };
    auto rshF = [&](unsigned b, F2 own) { return make_float2(own.y, lds<8>(b)); };
    auto lid2 = [&](F2 v, bool c0, bool c1) { return make_float2(c0 ? 0.f : v.x, c1 ? 0.f : v.y); };
    // ---- this thread's share of the radius-3 plane loads ----
    // nx % 4 == 0: one 16-byte chunk (4 columns of one row) per thread and
    // field.  Any other nx: 4-byte copies of plane elements t, t + NT, ...,
    // so that a warp reads 128 contiguous bytes and writes consecutive words.
    constexpr int NE = (PLL + L::NT - 1) / L::NT;
    const bool has_chunk = !LD && t < L::NCH;
    int ld_off = 0;
    bool z_all = false, z_u2 = false, patch_u1 = false;
    unsigned ld_dst = 0;
    int e_off[NE];
    unsigned e_dst[NE];  // shared word offset of each element (rows of pitch EX)
    unsigned e_flags = 0;
    if (a16) {
        if (has_chunk) {
            const int ey = t / L::CPR, cc = t % L::CPR;
            const int lx = x0 - 4 + 4 * cc, ly = y0 - 3 + ey;
            int cx, cy;
            bool outx = false, outy = false;
            if (perx) cx = wrap(lx, nx); else { outx = lx < 0 || lx >= nx; cx = outx ? 0 : lx; }
            if (pery) cy = wrap(ly, ny); else { outy = ly < 0 || ly >= ny; cy = outy ? 0 : ly; }
            z_all = outx || outy;
            z_u2 = z_all || (!pery && ly == 0);
            patch_u1 = LID && !perx && lx == 0;
            ld_off = cy * nx + cx;
            ld_dst = sm_base + (unsigned)(ey * EX + 4 * cc) * 4u;
        }
    } else {
#pragma unroll
        for (int r = 0; r < NE; ++r) {
            const int idx = t + r * L::NT;
            e_off[r] = 0;
            e_dst[r] = 0;
            if (idx < PLL) {
                const int lx = x0 - 4 + idx % EXL, ly = y0 - 3 + idx / EXL;
                e_dst[r] = (unsigned)((idx / EXL) * EX + idx % EXL);
                int cx, cy;
                bool outx = false, outy = false;
                if (perx) cx = wrap(lx, nx); else { outx = lx < 0 || lx >= nx; cx = outx ? 0 : lx; }
                if (pery) cy = wrap(ly, ny); else { outy = ly < 0 || ly >= ny; cy = outy ? 0 : ly; }
                e_off[r] = cy * nx + cx;
                e_flags |= (unsigned)(outx || outy) << (3 * r);
                e_flags |= (unsigned)(!pery && ly == 0) << (3 * r + 1);
                e_flags |= (unsigned)(LID && !perx && lx == 0) << (3 * r + 2);
            }
        }
    }
    // loads of plane p into ring byte offset so; an interior plane (E false)
    // needs no wrap, clamp or z-lid face
    auto issue = [&](auto Ec, int p, unsigned so) {
        constexpr bool E = decltype(Ec)::value;
        if (a16) {
            if (has_chunk) {
                const long long pz = E ? (long long)(perz ? wrap(p, nz) : min(max(p, 0), nz - 1)) : (long long)p;
                const long long pc = pz * nxy + ld_off;
                const bool zz = E && !perz && (p <= 0 || p >= nz);
                const unsigned d = ld_dst + so;
                static_assert(EX % 4 == 0, "rows must stay 16-byte aligned");
                cp16(d, psi + pc, z_all);
                cp16(d + FB, u1 + pc, z_all);
                cp16(d + 2 * FB, u2 + pc, z_u2);
                cp16(d + 3 * FB, u3 + pc, z_all || zz);
                cp16(d + 4 * FB, h + pc, z_all);
            }
        } else {
            const long long pz = (E ? (long long)(perz ? wrap(p, nz) : min(max(p, 0), nz - 1)) : (long long)p) * nxy;
            const bool zz = E && !perz && (p <= 0 || p >= nz);
            const unsigned d0 = sm_base + so;
#pragma unroll
            for (int r = 0; r < NE; ++r) {
                if (t + r * L::NT < PLL) {
                    const long long o = pz + e_off[r];
                    const unsigned d = d0 + e_dst[r] * 4u;
                    const bool ze = (e_flags >> (3 * r)) & 1u;
                    cp4(d, psi + o, ze);
                    cp4(d + FB, u1 + o, ze || ((e_flags >> (3 * r + 2)) & 1u));
                    cp4(d + 2 * FB, u2 + o, ze || ((e_flags >> (3 * r + 1)) & 1u));
                    cp4(d + 3 * FB, u3 + o, ze || zz);
                    cp4(d + 4 * FB, h + o, ze);
                }
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    const int p_first = perz ? -3 : -1;
    const int p_last = nz + 2;
    const int q1lo = perz ? -2 : 0, q1hi = perz ? nz + 1 : nz - 1;
    const int q1top = perz ? q1hi : nz;
    const int wlo = perz ? -2 : 0, whi = perz ? nz : nz - 2;
    const int vlo = perz ? -1 : 0, vhi = perz ? nz : nz - 1;

    const F2 Z = bc(0.f);
    F2 pn_mm = Z, pn_m = Z, pn_c = Z;
    F2 p1a = Z, p1b = Z, p1c = Z;
    F2 u1b = Z, u2b = Z, u3b = Z, hb = bc(1.f);
    F2 u1c = Z, u2c = Z, u3c = Z, hc = bc(1.f);
    F2 sxa = Z, sxb = Z, sya = Z, syb = Z;
    F2 wlo_v = Z, bu_prev = Z, bd_prev = Z, h_prev = bc(1.f);
    F2 dacc = Z, gx_own = Z, gy_own = Z;

    // Iteration p: alpha | beta | gamma as in pairs_tile.  K = (p - p_first) & 3
    // (or -1: from p at run time); E: check the z range of every stage.
    auto body = [&](auto Kc, auto Ec, const int p) {
        constexpr int K = decltype(Kc)::value;
        constexpr bool E = decltype(Ec)::value;
        const int q1 = p - 1, q2 = p - 2, q3 = p - 3;
        const int kk = K >= 0 ? K : ((p - p_first) & 3);
        const unsigned r2 = tb + (unsigned)(((kk + 2) & 3) * PB);   // ring, plane q2
        const unsigned r1 = tb + (unsigned)(((kk + 3) & 3) * PB);   // ring, plane q1
        const unsigned rp = tb + (unsigned)(kk * PB);               // ring, plane p
        const unsigned rp1 = tb + (unsigned)(((kk + 1) & 3) * PB);  // ring, plane p+1
        const unsigned b1 = tb + (unsigned)(((kk + 1) & 1) * PB);   // psi1/SX/SY slot of q1
        const unsigned b2 = tb + (unsigned)((kk & 1) * PB);         // ... of q2 (= of p)

        // ---- alpha ----
        if (in_out && (!E || (q3 >= 0 && q3 <= nz - 1))) {
            const F2 gxr = rshF(tb + oGX, gx_own), gyu = ldp<oGY + RB>(tb);
            dacc = add(add(sub(gxr, gx_own), sub(gyu, gy_own)), dacc);
        }
        F2 sxc = sxb, syc = syb, v1_own = Z, v2_own = Z, pl = Z, pd = Z, u1R = Z, u2U = Z;
        if (!E || (q1 >= q1lo && q1 <= q1top)) {
            sxc = add(lshC(b1 + oP1, p1c), p1c);
            syc = add(ldp<oP1 - RB>(b1), p1c);
            stp<oSX>(b1, sxc);
            stp<oSY>(b1, syc);
            stp<oSZ>(tb, add(p1b, p1c));
        }
        if (E && !perz && q1 == 0) { p1b = p1c; sxb = sxc; syb = syc; }
        if (in_v && (!E || (q2 >= vlo && q2 <= vhi))) {
            pl = lshF(b2 + oP1, p1b);
            pd = ldp<oP1 - RB>(b2);
            {
                u2U = ldp<2 * FB + RB>(r2);
                const F2 ua = add(add(add(lshF(r2 + 2 * FB, u2b), u2b),
                                      make_float2(lds<2 * FB + RB - 4>(r2), u2U.x)), u2U);
                const F2 ub = add(add(add(lshF(r2 + 3 * FB, u3b), u3b), lshF(r1 + 3 * FB, u3c)), u3c);
                const F2 v = pseudo_velocity(u1b, p1b, pl, sxb, ldU(b2 + oSX), ldD(b2 + oSX), ua, sxc, sxa,
                                             ub, add(lshF(r2 + 4 * FB, hb), hb), eps);
                v1_own = LID ? lid2(v, xlid0, xlid1) : v;
            }
            {
                const F2 u1D = ldp<FB - RB>(r2);
                const F2 va = add(add(add(ldp<3 * FB - RB>(r2), u3b), ldp<3 * FB - RB>(r1)), u3c);
                u1R = rshF(r2 + FB, u1b);
                const F2 vb = add(add(add(u1D, u1b), make_float2(u1D.y, lds<FB - RB + 8>(r2))), u1R);
                const F2 v = pseudo_velocity(u2b, p1b, pd, syb, syc, sya, va, rshC(b2 + oSY, syb),
                                             lshC(b2 + oSY, syb), vb, add(ldp<4 * FB - RB>(r2), hb), eps);
                v2_own = (LID && ylid) ? Z : v;
            }
            stp<oV1>(tb, v1_own);
            stp<oV2>(tb, v2_own);
        }
        __syncthreads();  // (F)

        // ---- beta ----
        F2 whi_v = Z, bu_c = Z, bd_c = Z;
        if (in_beta) {
            if (!E || (q2 >= wlo && q2 <= whi)) {
                const F2 szo = add(p1b, p1c);
                // the x/y pseudo-velocities (same z range when E is false) read
                // u1 right of the pair and u2 above it already
                const F2 u1R2 = !E ? u1R : rshF(r2 + FB, u1b);
                const F2 u2U2 = !E ? u2U : ldp<2 * FB + RB>(r2);
                const F2 ua = add(add(add(u1b, u1c), u1R2), rshF(r1 + FB, u1c));
                const F2 ub = add(add(add(u2b, u2c), u2U2), ldp<2 * FB + RB>(r1));
                whi_v = pseudo_velocity(u3c, p1c, p1b, szo, rshC(tb + oSZ, szo), lshC(tb + oSZ, szo), ua,
                                        ldU(tb + oSZ), ldD(tb + oSZ), ub, add(hb, hc), eps);
            }
            if (NONOSC && (!E || (q2 >= vlo && q2 <= vhi))) {
                const F2 aL = lshC(r2, pn_m), aR = rshC(r2, pn_m), aD = ldD(r2), aU = ldU(r2);
                // psi1's left and lower neighbours: pl and pd of the alpha phase
                // (same z range), clamped behind a lid
                const F2 bL = LID ? make_float2(clampL ? p1b.x : pl.x, p1b.x) : pl;
                const F2 bD = (LID && dD == 0) ? p1b : pd;
                const F2 bR = rshC(b2 + oP1, p1b), bU = ldU(b2 + oP1);
                F2 mx = max3(max3(aL, aR, aD), max3(aU, bL, bR), max3(bD, bU, pn_mm));
                mx = max3(mx, max3(pn_m, pn_c, p1a), max3(p1b, p1c, p1b));
                F2 mn = min3(min3(aL, aR, aD), min3(aU, bL, bR), min3(bD, bU, pn_mm));
                mn = min3(mn, min3(pn_m, pn_c, p1a), min3(p1b, p1c, p1b));
                const F2 v1h = rshF(tb + oV1, v1_own), v2h = ldp<oV2 + RB>(tb);
                const F2 in = add(add(sub(mul(pos(v1_own), bL), mul(neg(v1h), bR)),
                                      sub(mul(pos(v2_own), bD), mul(neg(v2h), bU))),
                                  sub(mul(pos(wlo_v), p1a), mul(neg(whi_v), p1c)));
                const F2 outf = mul(add(add(sub(pos(v1h), neg(v1_own)), sub(pos(v2h), neg(v2_own))),
                                        sub(pos(whi_v), neg(wlo_v))), p1b);
                bu_c = mul(mul(sub(mx, p1b), hb), rcp(add(in, eps)));
                bd_c = mul(mul(sub(p1b, mn), hb), rcp(add(outf, eps)));
                stp<oBU>(tb, bu_c);
                stp<oBD>(tb, bd_c);
            }
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // plane p+1 landed
        if (LID && !LD && patch_u1)
            sm[(ld_dst - sm_base) / 4u + (unsigned)(L::NR * PL + ((kk + 1) & 3) * PL)] = 0.f;
        __syncthreads();  // (H)
        // plane p+2 into the slot of q2, which no stage reads any more
        if (!LD && (!E || p + 2 <= p_last)) issue(Ec, p + 2, (unsigned)(((kk + 2) & 3) * PB));

        // ---- gamma ----
        if (in_vm && (!E || (q2 >= 0 && q2 <= nz - 1))) {
            F2 vm1 = v1_own, vm2 = v2_own;
            if (NONOSC) {
                const F2 buL = lshF(tb + oBU, bu_c), bdL = lshF(tb + oBD, bd_c);
                const F2 buD = ldp<oBU - RB>(tb), bdD = ldp<oBD - RB>(tb);
                const F2 one = bc(1.f);
                vm1 = add(mul(pos(v1_own), min3(one, bdL, bu_c)), mul(neg(v1_own), min3(one, buL, bd_c)));
                vm2 = add(mul(pos(v2_own), min3(one, bdD, bu_c)), mul(neg(v2_own), min3(one, buD, bd_c)));
            }
            gx_own = flux(vm1, pl, p1b);
            gy_own = flux(vm2, pd, p1b);
            if (LID) {
                gx_own = lid2(gx_own, xlid0, xlid1);
                gy_own = ylid ? Z : gy_own;
            }
            stp<oGX>(tb, gx_own);
            stp<oGY>(tb, gy_own);
        }
        const bool q3ok = !E || (q3 >= 0 && q3 <= nz - 1), q2ok = !E || (q2 >= 0 && q2 <= nz - 1);
        if (in_out && (q3ok || q2ok)) {
            F2 gz = Z;
            if (!E || perz || (q2 >= 1 && q2 <= nz - 1)) {
                F2 vm3 = wlo_v;
                if (NONOSC) {
                    const F2 one = bc(1.f);
                    vm3 = add(mul(pos(wlo_v), min3(one, bd_prev, bu_c)), mul(neg(wlo_v), min3(one, bu_prev, bd_c)));
                }
                gz = flux(vm3, p1a, p1b);
            }
            if (q3ok && store) {
                const F2 v = sub(p1a, mul(add(dacc, gz), rcp(h_prev)));
                float *const o = outp + (long long)q3 * nxy;
                if (a16) {
                    st2(o, v);
                } else {
                    o[0] = v.x;
                    if (gx + 1 < nx) o[1] = v.y;
                }
            }
            dacc = sub(Z, gz);
        }
        // (a1) donor pass at plane p
        F2 p1n = p1c;
        const F2 pn_p = ldp<0>(rp);
        const F2 u1p = ldp<FB>(rp), u2p = ldp<2 * FB>(rp), u3p = ldp<3 * FB>(rp), hp = ldp<4 * FB>(rp);
        if (!E || (p >= q1lo && p <= q1hi)) {
            const F2 pn_n = ldp<0>(rp1);
            const F2 u3n = ldp<3 * FB>(rp1);
            const F2 fxl = flux(u1p, lshC(rp, pn_p), pn_p);
            const F2 fxh = flux(rshF(rp + FB, u1p), pn_p, rshC(rp, pn_p));
            const F2 fyl = flux(u2p, ldD(rp), pn_p);
            const F2 fyh = flux(ldp<2 * FB + RB>(rp), pn_p, ldU(rp));
            const F2 fzl = flux(u3p, pn_c, pn_p);
            const F2 fzh = flux(u3n, pn_p, pn_n);
            const F2 div = add(add(sub(fxh, fxl), sub(fyh, fyl)), sub(fzh, fzl));
            p1n = sub(pn_p, mul(div, rcp(hp)));
        }
        if (!E || (p >= q1lo && p <= q1top)) stp<oP1>(b2, p1n);
        __syncthreads();  // (X)

        h_prev = hb;
        pn_mm = pn_m; pn_m = pn_c; pn_c = pn_p;
        u1b = u1c; u2b = u2c; u3b = u3c; hb = hc;
        u1c = u1p; u2c = u2p; u3c = u3p; hc = hp;
        p1a = p1b; p1b = p1c; p1c = p1n;
        sxa = sxb; sxb = sxc; sya = syb; syb = syc;
        wlo_v = whi_v; bu_prev = bu_c; bd_prev = bd_c;
    };

    if (!LD) {
        issue(BT(), p_first, 0u);
        issue(BT(), p_first + 1, (unsigned)PB);
    }
    const int n_iter = p_last - p_first + 1;
    // interior iterations 3 <= p <= nz - 3, in whole blocks of four starting
    // at an iteration index that is a multiple of four
    const int i_s = (3 - p_first + 3) & ~3;
    const int nblk = max(0, nz - 3 - p_first + 1 - i_s) >> 2;
#pragma unroll 1
    for (int i = 0; i < n_iter;) {
        if (i == i_s && nblk > 0) {
#pragma unroll 1
            for (int b = 0; b < nblk; ++b, i += 4) {
                const int p = p_first + i;
                body(IC<0>(), BF(), p);
                body(IC<1>(), BF(), p + 1);
                body(IC<2>(), BF(), p + 2);
                body(IC<3>(), BF(), p + 3);
            }
            continue;
        }
        body(IC<-1>(), BT(), p_first + i);
        ++i;
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
}

template <int TX, int TY, bool NONOSC, bool LID, int AL, bool LD = false>
__global__ void __launch_bounds__(LD ? Lay2<TX, TY>::NTW + Lay2<TX, TY>::NLD : Lay2<TX, TY>::NT, Lay2<TX, TY>::MINB)
    k_fused_pairs(TileArgs a) {
    extern __shared__ __align__(16) float sm[];
    pairs_tile<TX, TY, NONOSC, LID, AL, LD>(a, blockIdx.x, sm);
}

// Persistent batched launch: CTA c runs work items [begin[c], begin[c+1]) of
// the item list, each item a (grid, tile) pair; parity selects which buffer
// of each grid's (psi, scratch) pair is read.
template <int TX, int TY, bool NONOSC, bool LID, bool LD = false>
__global__ void __launch_bounds__(LD ? Lay2<TX, TY>::NTW + Lay2<TX, TY>::NLD : Lay2<TX, TY>::NT, 1)
    k_fused_pairs_batch(const BatchGrid *__restrict__ grids, const int2 *__restrict__ items,
                        const int *__restrict__ begin, int parity) {
    extern __shared__ __align__(16) float sm[];
    const int lo = begin[blockIdx.x], hi = begin[blockIdx.x + 1];
    for (int it = lo; it < hi; ++it) {
        const int2 w = items[it];
        pairs_tile<TX, TY, NONOSC, LID, LD ? 1 : 2, LD>(batch_args(grids[w.x], parity), w.y, sm);
    }
}

// Run of CTA c in a direct batch (uniform: every index is blockIdx-derived
// and every table sits in the parameter space).
__device__ __forceinline__ int direct_run(const DirectBatch &d, int c) {
    int lo = 0, hi = d.nruns;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (d.start[mid] <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int TX, int TY, bool NONOSC, bool LID, bool LD = false>
__global__ void __launch_bounds__(LD ? Lay2<TX, TY>::NTW + Lay2<TX, TY>::NLD : Lay2<TX, TY>::NT, 1)
    k_fused_pairs_direct(const __grid_constant__ DirectBatch d, int parity) {
    extern __shared__ __align__(16) float sm[];
    const int c = blockIdx.x, r = direct_run(d, c);
    pairs_tile<TX, TY, NONOSC, LID, LD ? 1 : 2, LD>(batch_args(d.g[r], parity), d.tile0[r] + c - d.start[r], sm);
}

// Loader warps serve the 12-, 24- and 28-row tiles of launches whose grids all
// have nx % 4 == 0 (16-byte loads); 16-row tiles and any other nx keep the
// compute threads' own loads.
template <int TY>
constexpr bool has_loaders() { return TY == 12 || TY == 24 || TY == 28; }

template <int TX, int TY>
constexpr int pairs_threads(bool ld) { return ld ? Lay2<TX, TY>::NTW + Lay2<TX, TY>::NLD : Lay2<TX, TY>::NT; }

template <int TX, int TY>
constexpr size_t pairs_smem() {  // the two-column kernel's 4-plane ring
    return (size_t)Lay2<TX, TY, 4>::NPLANES * Lay2<TX, TY, 4>::PL * sizeof(float);
}

using SingleKernel = void (*)(TileArgs);

template <int TX, int TY, int AL, bool LD>
SingleKernel single_kernel(int nonosc, bool lid) {
    return nonosc ? (lid ? k_fused_pairs<TX, TY, true, true, AL, LD> : k_fused_pairs<TX, TY, true, false, AL, LD>)
                  : (lid ? k_fused_pairs<TX, TY, false, true, AL, LD> : k_fused_pairs<TX, TY, false, false, AL, LD>);
}

template <int TX, int TY>
SingleKernel pick_single(const Grid &g, int nonosc, bool &ld) {
    const bool lid = !g.per[0] || !g.per[1];
    const bool a16 = g.nx % 4 == 0;
    ld = false;
    if (!a16) return single_kernel<TX, TY, 0, false>(nonosc, lid);
    if constexpr (has_loaders<TY>()) {
        ld = true;
        return single_kernel<TX, TY, 1, true>(nonosc, lid);
    } else {
        return single_kernel<TX, TY, 1, false>(nonosc, lid);
    }
}

// Tile rows [y0, y0 + TY * nty) of one grid in one launch.
template <int TX, int TY>
cudaError_t launch_rows(const PairsRows &r) {
    const size_t smem = pairs_smem<TX, TY>();
    bool ld;
    const SingleKernel kern = pick_single<TX, TY>(r.g, r.nonosc, ld);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && Lay2<TX, TY>::MINB > 1)  // room for MINB CTAs per SM
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    TileArgs a;
    a.g = r.g;
    a.ntx = (r.g.nx + TX - 1) / TX;
    a.y0 = r.y0;
    a.eps = (float)r.eps;
    a.h = (const float *)r.h; a.psi = (const float *)r.psi; a.u1 = (const float *)r.u1;
    a.u2 = (const float *)r.u2; a.u3 = (const float *)r.u3; a.out = (float *)r.out;
    kern<<<a.ntx * r.nty, pairs_threads<TX, TY>(ld), smem, r.s>>>(a);
    return cudaGetLastError();
}

template <int TX, int TY, bool LD>
cudaError_t launch_pairs_batch(int nonosc, int lid, const BatchGrid *grids, const int2 *items,
                               const int *begin, int ncta, int parity, cudaStream_t s) {
    const size_t smem = pairs_smem<TX, TY>();
    auto kern = nonosc ? (lid ? k_fused_pairs_batch<TX, TY, true, true, LD> : k_fused_pairs_batch<TX, TY, true, false, LD>)
                       : (lid ? k_fused_pairs_batch<TX, TY, false, true, LD> : k_fused_pairs_batch<TX, TY, false, false, LD>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ncta, pairs_threads<TX, TY>(LD), smem, s>>>(grids, items, begin, parity);
    return cudaGetLastError();
}

template <int TX, int TY, bool LD>
cudaError_t launch_pairs_direct(int nonosc, int lid, const DirectBatch &d, int parity, cudaStream_t s) {
    const size_t smem = pairs_smem<TX, TY>();
    auto kern = nonosc ? (lid ? k_fused_pairs_direct<TX, TY, true, true, LD> : k_fused_pairs_direct<TX, TY, true, false, LD>)
                       : (lid ? k_fused_pairs_direct<TX, TY, false, true, LD> : k_fused_pairs_direct<TX, TY, false, false, LD>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<d.start[d.nruns], pairs_threads<TX, TY>(LD), smem, s>>>(d, parity);
    return cudaGetLastError();
}

}  // namespace

// Entry points per tile height, one translation unit each
// (mpdata_fused2_t<TY>.cu), so that the kernel instances compile in
// parallel.  ld: the launch's grids all have nx % 4 == 0 and the tile takes
// its loader warps.
cudaError_t pairs_rows_t12(const PairsRows &r);
cudaError_t pairs_rows_t16(const PairsRows &r);
cudaError_t pairs_rows_t24(const PairsRows &r);
cudaError_t pairs_rows_t28(const PairsRows &r);
cudaError_t pairs_batch_t16(int ld, int nonosc, int lid, const BatchGrid *grids, const int2 *items,
                            const int *begin, int ncta, int parity, cudaStream_t s);
cudaError_t pairs_batch_t24(int ld, int nonosc, int lid, const BatchGrid *grids, const int2 *items,
                            const int *begin, int ncta, int parity, cudaStream_t s);
cudaError_t pairs_batch_t28(int ld, int nonosc, int lid, const BatchGrid *grids, const int2 *items,
                            const int *begin, int ncta, int parity, cudaStream_t s);
cudaError_t pairs_direct_t16(int ld, int nonosc, int lid, const DirectBatch &d, int parity, cudaStream_t s);
cudaError_t pairs_direct_t24(int ld, int nonosc, int lid, const DirectBatch &d, int parity, cudaStream_t s);
cudaError_t pairs_direct_t28(int ld, int nonosc, int lid, const DirectBatch &d, int parity, cudaStream_t s);

}  // namespace mpdata
