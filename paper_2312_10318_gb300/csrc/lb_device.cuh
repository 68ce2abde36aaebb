// Device side of the D2Q9 TRT-RLB library: lattice constants, the per-node
// collision (eq2 with eq4, eq6, eq9, eq11, eq_Gi) in D2Q9-reduced form, and the
// AA-pattern storage rules shared by every kernel.
//
// Storage.  Populations live in one array F[9][ny][pitch] (x fastest, pitch a
// multiple of 64 elements) as the shifted deviation d_i = f_i - w_i rho0 in
// the storage type S.  The AA pattern keeps one copy: for a state at an EVEN
// time level, f_i(x) sits at F[i][x]; at an ODD level it sits at
// F[ibar][x - e_i] when x - e_i is a streaming node (fluid or outlet ghost
// inside the domain), and at F[i][x] when x - e_i is a wall (bounce-back
// storage).  An even step reads and writes only a node's own slots (it writes
// f*_i to F[ibar][x]); an odd step reads the neighbour slots above and writes
// f*_i to F[i][x + e_i] (or F[ibar][x] at a wall), which are the same nine
// locations, so the update is in place and race-free.
#pragma once
#include <type_traits>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace trt {

// ---- D2Q9 (Sec. II B) -----------------------------------------------------
__host__ __device__ constexpr int ex(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5);
}
__host__ __device__ constexpr double wgt(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

enum : uint8_t { FLUID = 0, SOLID = 1, INLET = 2, OUTLET = 3, PRESSURE = 4, HALO = 5, HALO_PRESSURE = 6 };

// Classes whose nodes collide: fluid nodes and Zou-He pressure outlet nodes.
__host__ __device__ constexpr bool collides(int c) { return c == FLUID || c == PRESSURE; }
enum : int { K_STREAM = 0, K_WALL = 1, K_MOVING = 2 };
enum : int { G_LAGGED = 0, G_CURRENT = 1, G_OFF = 2 };

// ---- storage formats --------------------------------------------------------
template <typename S> struct Fmt;
template <> struct Fmt<double> {
    using C = double;
    static __device__ __forceinline__ double ld(double v) { return v; }
    static __device__ __forceinline__ double st(double v) { return v; }
};
template <> struct Fmt<float> {
    using C = float;
    static __device__ __forceinline__ float ld(float v) { return v; }
    static __device__ __forceinline__ float st(float v) { return v; }
};
template <> struct Fmt<__half> {
    using C = float;
    static __device__ __forceinline__ float ld(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half st(float v) { return __float2half_rn(v); }
};
template <> struct Fmt<__nv_bfloat16> {
    using C = float;
    static __device__ __forceinline__ float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};
}  // namespace trt
#include "lb_dw.cuh"   // FP64 storage with double-word FP32 arithmetic (Fmt<f64dw>)
namespace trt {

// ---- kernel arguments -------------------------------------------------------
template <typename C> struct Args {
    void* f;              // S[9][ny][pitch]
    const C* phi_in;      // [2][ny][pitch]: Phi of the previous level
    C* phi_out;           // [2][ny][pitch]: Phi of this level
    const uint8_t* mask;  // [ny][pitch] or nullptr
    const uint8_t* seg;   // [ny][segs]: 1 where a 32-node row segment and its neighbours are plain fluid
    int segs;
    int nx, ny, pitch;
    long long plane;      // ny * pitch
    int px, py;           // periodic flags
    C k1, k1lo, k2, k2lo; // 1 - 1/tau as a hi + lo pair (lo = 0 for FP64)
    C kf;                 // 1 - 1/(2 tau1)
    C gx, gy, rho0;
    C corr[9];            // moving-wall term 2 w_i rho_w (e_i.u_w) / c_s^2
    C phin_x, phin_y;     // Phi of moving-wall (inlet) nodes, rho_w u_w^3
    C zh_dr;              // rho0 - outlet_rho of the Zou-He pressure outlet
};

// Zou-He constant-pressure outlet (Sec. III D) on the shifted populations
// d_i = f_i - w_i rho0 of a node on the last column of a lattice open in x:
// the three populations entering across the edge (e_x = -1) are rebuilt so
// that rho = outlet_rho, rho u_y = 0 and the normal non-equilibrium parts of
// f_(1,0) and f_(-1,0) are equal.  With j = rho_out u_x =
// [d_0 + d_2 + d_4 + 2 (d_1 + d_5 + d_8)] + (rho0 - rho_out) (the weights of
// f_0 + f_2 + f_4 + 2 (f_1 + f_5 + f_8) add up to 1):
//   d_3 = d_1 - (2/3) j,  d_6 = d_8 - (d_2 - d_4)/2 - j/6,
//   d_7 = d_5 + (d_2 - d_4)/2 - j/6.
template <typename C>
__device__ __forceinline__ void zh_fill(C (&d)[9], C zh_dr) {
    const C j = (d[0] + d[2] + d[4]) + C(2) * (d[1] + d[5] + d[8]) + zh_dr;
    const C t = C(0.5) * (d[2] - d[4]);
    const C j6 = j * C(1.0 / 6.0);
    d[3] = d[1] - C(4) * j6;
    d[6] = d[8] - t - j6;
    d[7] = d[5] + t - j6;
}

// Neighbourhood of node (x, y): wrapped coordinates and out-of-domain flags.
struct Nbh {
    int xm, xp, ym, yp;
    bool oxm, oxp, oym, oyp;
};

template <typename C>
__device__ __forceinline__ Nbh neighbours(const Args<C>& a, int x, int y) {
    Nbh n;
    n.xm = x - 1; n.xp = x + 1; n.ym = y - 1; n.yp = y + 1;
    n.oxm = n.oxp = n.oym = n.oyp = false;
    if (n.xm < 0) { if (a.px) n.xm += a.nx; else n.oxm = true; }
    if (n.xp >= a.nx) { if (a.px) n.xp -= a.nx; else n.oxp = true; }
    if (n.ym < 0) { if (a.py) n.ym += a.ny; else n.oym = true; }
    if (n.yp >= a.ny) { if (a.py) n.yp -= a.ny; else n.oyp = true; }
    return n;
}

// Linear index (within a plane, < 2^30) of x + e_i and whether it lies outside.
template <int I>
__device__ __forceinline__ int nb_index(const Nbh& n, int x, int y, int pitch, bool& out) {
    constexpr int dx = ex(I), dy = ey(I);
    const int cx = dx > 0 ? n.xp : (dx < 0 ? n.xm : x);
    const int cy = dy > 0 ? n.yp : (dy < 0 ? n.ym : y);
    out = (dx > 0 && n.oxp) || (dx < 0 && n.oxm) || (dy > 0 && n.oyp) || (dy < 0 && n.oym);
    return cy * pitch + cx;
}

__device__ __forceinline__ int kind_of(uint8_t c) {
    return c == SOLID ? K_WALL : (c == INLET ? K_MOVING : K_STREAM);
}

// Neighbourhood of a node of a lattice periodic in x and y (no flags needed).
template <typename C>
__device__ __forceinline__ Nbh neighbours_periodic(const Args<C>& a, int x, int y) {
    Nbh n;
    n.xm = x == 0 ? a.nx - 1 : x - 1;
    n.xp = x == a.nx - 1 ? 0 : x + 1;
    n.ym = y == 0 ? a.ny - 1 : y - 1;
    n.yp = y == a.ny - 1 ? 0 : y + 1;
    n.oxm = n.oxp = n.oym = n.oyp = false;
    return n;
}

// Link kinds of the 8 neighbours x + e_i (index 0 unused) and their indices.
template <bool GENERAL, typename C>
__device__ __forceinline__ void links(const Args<C>& a, int x, int y, int (&nb)[9],
                                      int (&kind)[9]) {
    const Nbh n = GENERAL ? neighbours(a, x, y) : neighbours_periodic(a, x, y);
    bool out[9];
    nb[0] = y * a.pitch + x;
    kind[0] = K_STREAM;
    out[0] = false;
#define TRT_NB(I) nb[I] = nb_index<I>(n, x, y, a.pitch, out[I]);
    TRT_NB(1) TRT_NB(2) TRT_NB(3) TRT_NB(4) TRT_NB(5) TRT_NB(6) TRT_NB(7) TRT_NB(8)
#undef TRT_NB
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        if (!GENERAL) {
            kind[i] = K_STREAM;
        } else if (out[i]) {
            kind[i] = K_WALL;
        } else {
            kind[i] = a.mask ? kind_of(a.mask[nb[i]]) : K_STREAM;
        }
    }
}

// Location (offset into F) of f_i(x, t) for a state whose level has parity ODD.
template <bool ODD>
__device__ __forceinline__ long long pop_loc(long long plane, const int (&nb)[9],
                                             const int (&kind)[9], int i) {
    if (!ODD) return (long long)i * plane + nb[0];
    const int j = opp(i);  // x - e_i = x + e_j
    return kind[j] == K_STREAM ? (long long)j * plane + nb[j] : (long long)i * plane + nb[0];
}

// ---- the collision ----------------------------------------------------------
// d: shifted pre-collision populations d_i = f_i - w_i rho0 of one node.
// dpx = d_x Phi_xxx, dpy = d_y Phi_yyy (central differences, already halved).
// o: shifted post-collision populations f*_i - w_i rho0, the right-hand side
// of eq2.  In D2Q9 every Hermite contraction collapses: with
//   a1 = j + F,
//   a2_ab = rho u_a u_b + (1 - 1/tau1) A_ab + (1 - 1/(2 tau1))(F_a u_b + u_a F_b)
//           - (1 - 1/(2 tau1)) d_g Phi_abg   (rho u_a u_b + A_ab = sum H_ab f),
//   a3_xxy = rho u_x^2 u_y + (1 - 1/tau2) A_xxy  (and xyy alike),
// f*_i = w_i [rho + 3 e_i.a1 + 9/2 H_i,ab a2_ab + 27/2 (H_i,xxy a3_xxy +
// H_i,xyy a3_xyy)], because 1/(2 c_s^4) = 1/(6 c_s^6) = 9/2, H_xxx = H_yyy = 0
// and the first-order terms of eq2 combine into w_i e_i.(j + F)/c_s^2.  The
// weights w_i are folded into the coefficients below.  The raw moments share
// their partial sums (the compiler may not reassociate float additions).
// Returns Phi_xxx = rho u_x^3 and Phi_yyy = rho u_y^3 of the node (eq11 u).
//
// collide_dw: the same collision for double-word pairs, arranged for fewer
// double-word operations (each costs 8-11 FP32 instructions, and this format
// is bound by them): scalings by powers of two are exact per component, the
// reconstruction shares b9 = drho/9, h = a2/3 and g = a1/3 (5 products by
// constants instead of 16), the reciprocal is taken directly, and without a
// body force (a uniform branch) the forcing terms are skipped -- they would
// add exact zeros.
__device__ __forceinline__ df64 scale2(const df64& x, float p) {   // p a power of two
    return df64(__fmul_rn(x.hi, p), __fmul_rn(x.lo, p));
}

__device__ __forceinline__ void collide_dw(const df64 (&d)[9], df64 dpx, df64 dpy, const df64 k1,
                                           const df64 k2, const df64 kf, const df64 gx,
                                           const df64 gy, const df64 rho0, df64 (&o)[9], df64& phx,
                                           df64& phy) {
    const df64 third = df64(1.0 / 3.0);
    const df64 s13 = d[1] + d[3], m13 = d[1] - d[3];
    const df64 s24 = d[2] + d[4], m24 = d[2] - d[4];
    const df64 a57 = d[5] + d[7], m57 = d[5] - d[7];
    const df64 a68 = d[6] + d[8], m68 = d[6] - d[8];
    const df64 sd = a57 + a68, pxy = a57 - a68;
    const df64 qxxy = m57 + m68, qxyy = m57 - m68;
    const df64 jx = m13 + qxyy, jy = m24 + qxxy;
    const df64 drho = (d[0] + sd) + (s13 + s24);
    const df64 rho = rho0 + drho;
    const df64 inv = recip(rho);
    const bool forced = gx.hi != 0.f || gx.lo != 0.f || gy.hi != 0.f || gy.lo != 0.f;
    df64 ux = jx * inv, uy = jy * inv;
    if (forced) {
        ux = ux + scale2(gx, 0.5f);
        uy = uy + scale2(gy, 0.5f);
    }
    const df64 rux = rho * ux, ruy = rho * uy;
    const df64 ruxx = rux * ux, ruyy = ruy * uy, ruxy = rux * uy;
    const df64 rxxy = ruxx * uy, rxyy = ruyy * ux;
    const df64 drho3 = third * drho;
    const df64 Axx = ((s13 + sd) - drho3) - ruxx, Ayy = ((s24 + sd) - drho3) - ruyy;
    const df64 Axy = pxy - ruxy;
    const df64 Axxy = (qxxy - third * jy) - rxxy, Axyy = (qxyy - third * jx) - rxyy;
    df64 a1x = jx, a1y = jy;
    df64 a2xx = (ruxx + k1 * Axx) - kf * dpx;
    df64 a2yy = (ruyy + k1 * Ayy) - kf * dpy;
    df64 a2xy = ruxy + k1 * Axy;
    if (forced) {
        const df64 Fx = rho * gx, Fy = rho * gy;
        a1x = a1x + Fx;
        a1y = a1y + Fy;
        a2xx = a2xx + kf * scale2(Fx * ux, 2.f);
        a2yy = a2yy + kf * scale2(Fy * uy, 2.f);
        a2xy = a2xy + kf * (Fx * uy + ux * Fy);
    }
    const df64 a3xxy = rxxy + k2 * Axxy, a3xyy = rxyy + k2 * Axyy;
    // reconstruction with the weights folded in (see collide)
    const df64 b9 = third * drho3;                   // drho / 9
    const df64 hxx = third * a2xx, hyy = third * a2yy;
    const df64 g1x = third * a1x, g1y = third * a1y;
    const df64 ht = hxx + hyy;                       // (a2xx + a2yy) / 3
    o[0] = scale2(b9, 4.f) - scale2(ht, 2.f);
    const df64 c13 = (b9 + hxx) - scale2(hyy, 0.5f);
    const df64 c24 = (b9 + hyy) - scale2(hxx, 0.5f);
    const df64 o13 = g1x - scale2(a3xyy, 0.5f);
    const df64 o24 = g1y - scale2(a3xxy, 0.5f);
    o[1] = c13 + o13;
    o[3] = c13 - o13;
    o[2] = c24 + o24;
    o[4] = c24 - o24;
    const df64 cd = scale2(b9 + ht, 0.25f);
    const df64 q = scale2(a2xy, 0.25f);
    const df64 c57 = cd + q, c68 = cd - q;
    const df64 o57 = scale2((g1x + g1y) + (a3xxy + a3xyy), 0.25f);
    const df64 o68 = scale2((g1y - g1x) + (a3xxy - a3xyy), 0.25f);
    o[5] = c57 + o57;
    o[7] = c57 - o57;
    o[6] = c68 + o68;
    o[8] = c68 - o68;
    phx = ruxx * ux;
    phy = ruyy * uy;
}

// Raw moments of one node's shifted populations and its eq11 velocity: the
// first half of the collision, which the two-buffer TMA kernel also uses for
// Phi before its halo barrier.
template <typename C> struct NodeMom {
    C drho, s13, s24, sd, pxy, qxxy, qxyy, jx, jy;   // sums of d weighted by e
    C rho, ux, uy;
};

template <typename C>
__device__ __forceinline__ NodeMom<C> node_moments(const C (&d)[9], const C gx, const C gy,
                                                   const C rho0) {
    NodeMom<C> m;
    m.s13 = d[1] + d[3];
    const C m13 = d[1] - d[3];
    m.s24 = d[2] + d[4];
    const C m24 = d[2] - d[4];
    const C a57 = d[5] + d[7], m57 = d[5] - d[7];
    const C a68 = d[6] + d[8], m68 = d[6] - d[8];
    m.sd = a57 + a68;      // sum of the four diagonal populations
    m.pxy = a57 - a68;     // sum e_x e_y d
    m.qxxy = m57 + m68;    // sum e_x^2 e_y d
    m.qxyy = m57 - m68;    // sum e_x e_y^2 d
    m.jx = m13 + m.qxyy;   // sum e_x d
    m.jy = m24 + m.qxxy;   // sum e_y d
    m.drho = (d[0] + m.sd) + (m.s13 + m.s24);
    // eq11: rho = sum f, u = (sum e f)/rho + g/2
    m.rho = rho0 + m.drho;
    const C inv = C(1) / m.rho;
    m.ux = m.jx * inv + C(0.5) * gx;
    m.uy = m.jy * inv + C(0.5) * gy;
    return m;
}

// The rest of the collision (eq2 with eq9, eq_Gi and eq6) from the moments.
template <typename C>
__device__ __forceinline__ void collide_from(const NodeMom<C>& m, C dpx, C dpy, const C k1,
                                             const C k1lo, const C k2, const C k2lo, const C kf,
                                             const C gx, const C gy, C (&o)[9], C& phx, C& phy) {
    const C third = C(1.0 / 3.0);
    const C drho = m.drho, rho = m.rho, ux = m.ux, uy = m.uy, jx = m.jx, jy = m.jy;
    const C Fx = rho * gx, Fy = rho * gy;
    const C rux = rho * ux, ruy = rho * uy;
    const C ruxx = rux * ux, ruyy = ruy * uy, ruxy = rux * uy;
    const C rxxy = ruxx * uy, rxyy = ruyy * ux;
    // Hermite moments sum H f: second order (H_xx = e_x^2 - 1/3, ...) and the
    // surviving third-order components; minus the equilibrium moments of
    // eq9_2 they are the non-equilibrium projections A of eq9 (A_x = -F_x/2
    // is folded into a1)
    const C drho3 = third * drho;
    const C Pxx = (m.s13 + m.sd) - drho3, Pyy = (m.s24 + m.sd) - drho3;
    const C Qxxy = m.qxxy - third * jy, Qxyy = m.qxyy - third * jx;
    const C Axx = Pxx - ruxx, Ayy = Pyy - ruyy, Axy = m.pxy - ruxy;
    const C Axxy = Qxxy - rxxy, Axyy = Qxyy - rxyy;
    // relaxation: (1 - 1/tau) A with 1 - 1/tau carried as hi + lo, so the rate
    // 1/tau stays exact to ~2^-48 even when tau is large (FP32 alone would
    // round 1 - 1/tau to 2^-24 absolute, i.e. 1/tau to 2^-24 tau relative)
    // (FP64 needs no low part: its rounding of 1 - 1/tau is below 1e-11 of the
    // rate for any tau this library accepts in practice)
    constexpr bool split = sizeof(C) < 8;
    const C a1x = jx + Fx, a1y = jy + Fy;
    C r2xx = ruxx + k1 * Axx, r2yy = ruyy + k1 * Ayy, r2xy = ruxy + k1 * Axy;
    C a3xxy = rxxy + k2 * Axxy, a3xyy = rxyy + k2 * Axyy;
    if (split) {
        r2xx += k1lo * Axx;
        r2yy += k1lo * Ayy;
        r2xy += k1lo * Axy;
        a3xxy += k2lo * Axxy;
        a3xyy += k2lo * Axyy;
    }
    const C a2xx = r2xx + kf * (C(2) * Fx * ux - dpx);
    const C a2yy = r2yy + kf * (C(2) * Fy * uy - dpy);
    const C a2xy = r2xy + kf * (Fx * uy + ux * Fy);
    // reconstruction, w_i folded in: w0 = 4/9, w1..4 = 1/9, w5..8 = 1/36
    const C t = a2xx + a2yy;
    o[0] = C(4.0 / 9.0) * drho - C(2.0 / 3.0) * t;
    const C b9 = C(1.0 / 9.0) * drho;
    const C c13 = b9 + C(1.0 / 3.0) * a2xx - C(1.0 / 6.0) * a2yy;
    const C o13 = C(1.0 / 3.0) * a1x - C(0.5) * a3xyy;
    const C c24 = b9 - C(1.0 / 6.0) * a2xx + C(1.0 / 3.0) * a2yy;
    const C o24 = C(1.0 / 3.0) * a1y - C(0.5) * a3xxy;
    o[1] = c13 + o13;
    o[3] = c13 - o13;
    o[2] = c24 + o24;
    o[4] = c24 - o24;
    const C cd = C(1.0 / 36.0) * drho + C(1.0 / 12.0) * t;
    const C q = C(0.25) * a2xy;
    const C c57 = cd + q, c68 = cd - q;
    const C o57 = C(1.0 / 12.0) * (a1x + a1y) + C(0.25) * (a3xxy + a3xyy);
    const C o68 = C(1.0 / 12.0) * (a1y - a1x) + C(0.25) * (a3xxy - a3xyy);
    o[5] = c57 + o57;
    o[7] = c57 - o57;
    o[6] = c68 + o68;
    o[8] = c68 - o68;
    phx = ruxx * ux;
    phy = ruyy * uy;
}

template <typename C>
__device__ __forceinline__ void collide(const C (&d)[9], C dpx, C dpy, const C k1, const C k1lo,
                                        const C k2, const C k2lo, const C kf, const C gx,
                                        const C gy, const C rho0, C (&o)[9], C& phx, C& phy) {
    if constexpr (std::is_same<C, df64>::value) {
        collide_dw(d, dpx, dpy, k1, k2, kf, gx, gy, rho0, o, phx, phy);
    } else {
        collide_from<C>(node_moments<C>(d, gx, gy, rho0), dpx, dpy, k1, k1lo, k2, k2lo, kf, gx, gy, o,
                        phx, phy);
    }
}

// Moments of one node from shifted populations (eq11).
template <typename C>
__device__ __forceinline__ void moments_of(const C (&d)[9], C gx, C gy, C rho0, C& rho, C& ux,
                                           C& uy) {
    const C drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    const C jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    const C jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    rho = rho0 + drho;
    const C inv = C(1) / rho;
    ux = jx * inv + C(0.5) * gx;
    uy = jy * inv + C(0.5) * gy;
}

// ---- kernels ----------------------------------------------------------------

// Resident 256-thread CTAs per SM the scalar step kernels ask the compiler to
// allow: the FP32 periodic step with lagged G fits 40 registers without
// spilling (6 CTAs, 75 % occupancy for the odd step instead of 5), the
// periodic double-word step 64 (4 CTAs; the odd step took 79 and 3).  The
// general steps (walls, masks, open edges) run the periodic code on interior
// row segments, so their own code may spill a little: FP32 and 16-bit 6 CTAs
// (40 registers; 12-80 bytes of spills in the boundary code), double-word 4
// (64 registers, no spills with Phi lagged).  Measured on 4096 x 2048 creeping
// flow and a 4096^2 channel (ms per step, compiler's choice / these): FP32
// 0.1635 / 0.1442 and 0.2984 / 0.2630, FP16 0.1316 / 0.1138 and 0.2367 /
// 0.2017, F64_DW 0.3826 / 0.3335 and 0.8070 / 0.7076 (3 CTAs: 0.3587 and
// 0.7563).  The other variants keep the compiler's choice.
template <typename S, bool GENERAL, int GMODE>
__host__ __device__ constexpr int step_min_blocks() {
    return (sizeof(S) == 4 && !GENERAL && GMODE == G_LAGGED) ? 6
           : (sizeof(S) <= 4 && GENERAL)                          ? 6
           : (std::is_same<S, f64dw>::value && !GENERAL)          ? 4
           : (std::is_same<S, f64dw>::value && GENERAL)           ? 4
                                                                   : 1;
}

// The periodic step (node_step_periodic, below) in two halves, for the general
// step's interior segments (the periodic kernels keep the single body, which
// compiles to a faster schedule).  The reads: the nine slots and, with Phi
// lagged, the two Phi differences.  Every index stays inside the buffers for any node of the
// lattice (the wrap corrections keep it in its plane), which the general step
// relies on when it issues these loads before it knows whether the node is
// interior.
template <typename S, bool ODD, int GMODE>
__device__ __forceinline__ void periodic_load(const Args<typename Fmt<S>::C>& a, int x, int y,
                                              typename Fmt<S>::C (&d)[9], typename Fmt<S>::C& dpx,
                                              typename Fmt<S>::C& dpy) {
    using C = typename Fmt<S>::C;
    const int own = y * a.pitch + x;
    const int pt = a.pitch;
    const int pl = (int)a.plane;           // a plane holds at most 2^30 nodes
    const int cxp = x == a.nx - 1 ? -a.nx : 0, cxm = x == 0 ? a.nx : 0;
    const int cyp = y == a.ny - 1 ? -pl : 0, cym = y == 0 ? pl : 0;
    const S* __restrict__ F = static_cast<const S*>(a.f);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int k = ODD ? opp(i) : i;
        int idx = own;
        if (ODD) {
            idx += ey(k) * pt + ex(k);
            idx += ex(k) > 0 ? cxp : (ex(k) < 0 ? cxm : 0);
            idx += ey(k) > 0 ? cyp : (ey(k) < 0 ? cym : 0);
        }
        d[i] = Fmt<S>::ld(F[(long long)k * a.plane + idx]);
    }
    dpx = C(0);
    dpy = C(0);
    if (GMODE == G_LAGGED) {
        const C* Px = a.phi_in + own;
        const C* Py = a.phi_in + a.plane + own;
        dpx = C(0.5) * (Px[1 + cxp] - Px[-1 + cxm]);
        dpy = C(0.5) * (Py[pt + cyp] - Py[-pt + cym]);
    }
}

// Its collision and writes, from the values periodic_load read.
template <typename S, bool ODD, int GMODE>
__device__ __forceinline__ void periodic_finish(const Args<typename Fmt<S>::C>& a, int x, int y,
                                                const typename Fmt<S>::C (&d)[9], typename Fmt<S>::C dpx,
                                                typename Fmt<S>::C dpy) {
    using C = typename Fmt<S>::C;
    const int own = y * a.pitch + x;
    const int pt = a.pitch;
    const int pl = (int)a.plane;
    const int cxp = x == a.nx - 1 ? -a.nx : 0, cxm = x == 0 ? a.nx : 0;
    const int cyp = y == a.ny - 1 ? -pl : 0, cym = y == 0 ? pl : 0;
    S* __restrict__ F = static_cast<S*>(a.f);
    C o[9], phx, phy;
    collide<C>(d, dpx, dpy, a.k1, a.k1lo, a.k2, a.k2lo, a.kf, a.gx, a.gy, a.rho0, o, phx, phy);
    if (GMODE == G_LAGGED) {
        a.phi_out[own] = phx;
        a.phi_out[a.plane + own] = phy;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int k = ODD ? i : opp(i);
        int idx = own;
        if (ODD) {
            idx += ey(k) * pt + ex(k);
            idx += ex(k) > 0 ? cxp : (ex(k) < 0 ? cxm : 0);
            idx += ey(k) > 0 ? cyp : (ey(k) < 0 ? cym : 0);
        }
        F[(long long)k * a.plane + idx] = Fmt<S>::st(o[i]);
    }
}

// The step of a node of a lattice periodic in x and y, without a mask.  The
// nine slots it reads and writes are A_k = F[k][x + e_k] on an odd level (it
// reads f_i from A_ibar and writes f*_i to A_i) and F[k][x] on an even one
// (reads f_i from F[i][x], writes f*_i to F[ibar][x]).  Each is the node's own
// index plus the offset k plane + e_yk pitch + e_xk, which is the same for
// every node, plus a wrap correction that is zero away from the lattice's
// edges: -nx for e_xk = 1 on the last column, +nx for e_xk = -1 on the first,
// -+ plane for e_yk = +-1 on the last and first rows.  No neighbour index is
// formed per access.
template <typename S, bool ODD, int GMODE>
__device__ __forceinline__ void node_step_periodic(const Args<typename Fmt<S>::C>& a, int x, int y) {
    using C = typename Fmt<S>::C;
    const int own = y * a.pitch + x;
    const int pt = a.pitch;
    const int pl = (int)a.plane;           // a plane holds at most 2^30 nodes
    const int cxp = x == a.nx - 1 ? -a.nx : 0, cxm = x == 0 ? a.nx : 0;
    const int cyp = y == a.ny - 1 ? -pl : 0, cym = y == 0 ? pl : 0;
    S* __restrict__ F = static_cast<S*>(a.f);
    C d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int k = ODD ? opp(i) : i;
        int idx = own;
        if (ODD) {
            idx += ey(k) * pt + ex(k);
            idx += ex(k) > 0 ? cxp : (ex(k) < 0 ? cxm : 0);
            idx += ey(k) > 0 ? cyp : (ey(k) < 0 ? cym : 0);
        }
        d[i] = Fmt<S>::ld(F[(long long)k * a.plane + idx]);
    }
    C dpx = C(0), dpy = C(0);
    if (GMODE == G_LAGGED) {
        const C* Px = a.phi_in + own;
        const C* Py = a.phi_in + a.plane + own;
        dpx = C(0.5) * (Px[1 + cxp] - Px[-1 + cxm]);
        dpy = C(0.5) * (Py[pt + cyp] - Py[-pt + cym]);
    }
    C o[9], phx, phy;
    collide<C>(d, dpx, dpy, a.k1, a.k1lo, a.k2, a.k2lo, a.kf, a.gx, a.gy, a.rho0, o, phx, phy);
    if (GMODE == G_LAGGED) {
        a.phi_out[own] = phx;
        a.phi_out[a.plane + own] = phy;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int k = ODD ? i : opp(i);
        int idx = own;
        if (ODD) {
            idx += ey(k) * pt + ex(k);
            idx += ex(k) > 0 ? cxp : (ex(k) < 0 ? cxm : 0);
            idx += ey(k) > 0 ? cyp : (ey(k) < 0 ? cym : 0);
        }
        F[(long long)k * a.plane + idx] = Fmt<S>::st(o[i]);
    }
}

// One fused AA step of one node (pull-stream, moments, regularized TRT
// collision, G_i, F_i, push-back into the same slots, half-way bounce-back);
// non-fluid nodes return at once.  GENERAL enables walls, masks and
// non-periodic edges; GMODE is G_LAGGED or G_OFF.
template <typename S, bool ODD, bool GENERAL, int GMODE>
__device__ __forceinline__ void node_step(const Args<typename Fmt<S>::C>& a, int x, int y) {
    using C = typename Fmt<S>::C;
    if constexpr (!GENERAL) {
        node_step_periodic<S, ODD, GMODE>(a, x, y);
        return;
    }
    // a row segment whose nodes and their neighbours are all plain fluid (no
    // wall, mask class or open edge on any link; a warp is one segment, so
    // the branch is uniform): the periodic step's code, same arithmetic.  Its
    // loads are issued together with the segment map's byte, not after it (they
    // stay inside the buffers for any node; elsewhere their values are unused)
    // (FP32 and 16-bit; the double-word step, issue-bound, measured faster
    // branching first)
    if (a.seg) {
        if constexpr (sizeof(S) <= 4) {
            const bool interior = a.seg[y * a.segs + (x >> 5)] != 0;
            C dq[9], dpxq, dpyq;
            periodic_load<S, ODD, GMODE>(a, x, y, dq, dpxq, dpyq);
            if (interior) {
                periodic_finish<S, ODD, GMODE>(a, x, y, dq, dpxq, dpyq);
                return;
            }
        } else if (a.seg[y * a.segs + (x >> 5)]) {
            node_step_periodic<S, ODD, GMODE>(a, x, y);
            return;
        }
    }
    S* __restrict__ F = static_cast<S*>(a.f);
    const int own = y * a.pitch + x;   // in-plane offsets stay below 2^30
    const int cls = (GENERAL && a.mask) ? a.mask[own] : FLUID;
    if (GENERAL && !collides(cls)) return;
    int nb[9];
    int kind[9];
    links<GENERAL>(a, x, y, nb, kind);

    C d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = Fmt<S>::ld(F[pop_loc<ODD>(a.plane, nb, kind, i)]);
    if (GENERAL && cls == PRESSURE) zh_fill<C>(d, a.zh_dr);

    C dpx = C(0), dpy = C(0);
    if (GMODE == G_LAGGED) {
        const Nbh n = GENERAL ? neighbours(a, x, y) : neighbours_periodic(a, x, y);
        const C* Px = a.phi_in;
        const C* Py = a.phi_in + a.plane;
        // beyond a pressure outlet Phi continues with zero gradient
        const C pxp = (GENERAL && n.oxp) ? (cls == PRESSURE ? Px[own] : C(0))
                                         : Px[y * a.pitch + n.xp];
        const C pxm = (GENERAL && n.oxm) ? C(0) : Px[y * a.pitch + n.xm];
        const C pyp = (GENERAL && n.oyp) ? C(0) : Py[n.yp * a.pitch + x];
        const C pym = (GENERAL && n.oym) ? C(0) : Py[n.ym * a.pitch + x];
        dpx = C(0.5) * (pxp - pxm);
        dpy = C(0.5) * (pyp - pym);
    }
    C o[9], phx, phy;
    collide<C>(d, dpx, dpy, a.k1, a.k1lo, a.k2, a.k2lo, a.kf, a.gx, a.gy, a.rho0, o, phx, phy);
    if (GMODE == G_LAGGED) {
        a.phi_out[own] = phx;
        a.phi_out[a.plane + own] = phy;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        C v = o[i];
        if (GENERAL && kind[i] == K_MOVING) v -= a.corr[i];
        long long dst;
        if (!ODD || kind[i] != K_STREAM)
            dst = (long long)opp(i) * a.plane + own;
        else
            dst = (long long)i * a.plane + nb[i];
        F[dst] = Fmt<S>::st(v);
    }
}

template <typename S, bool ODD, bool GENERAL, int GMODE>
__global__ void __launch_bounds__(256, step_min_blocks<S, GENERAL, GMODE>()) k_step(Args<typename Fmt<S>::C> a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    node_step<S, ODD, GENERAL, GMODE>(a, x, y);
}

// Outlet ghosts, after a step that produced a state of parity ODD_NEW: every
// population that a ghost s emits into a fluid node x = s + e_i is set to the
// post-collision f*_i of the inward neighbour z = s - (1, 0); Phi(s) := Phi(z).
template <typename S, bool ODD_NEW>
__global__ void k_ghosts(Args<typename Fmt<S>::C> a, const int* __restrict__ ghosts, int nghost) {
    using C = typename Fmt<S>::C;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nghost) return;
    S* F = static_cast<S*>(a.f);
    const int s = ghosts[g];
    const int sx = s % a.pitch, sy = s / a.pitch;
    int zx = sx - 1;
    if (zx < 0) zx += a.nx;  // validated: inside the domain (periodic) and fluid
    int nbs[9], nbz[9];
    int ks[9], kz[9];
    links<true>(a, sx, sy, nbs, ks);
    links<true>(a, zx, sy, nbz, kz);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        if (ks[i] != K_STREAM || !collides(a.mask[nbs[i]])) continue;
        // where the step stored f*_i(z)
        long long src;
        if (!ODD_NEW) {  // state is even: f*_i(z) went to F[i][z + e_i] or F[ibar][z]
            src = kz[i] == K_STREAM ? (long long)i * a.plane + nbz[i]
                                    : (long long)opp(i) * a.plane + nbz[0];
        } else {         // state is odd: an even step wrote f*_i(z) to F[ibar][z]
            src = (long long)opp(i) * a.plane + nbz[0];
        }
        // location of f_i(x) in the new state, x = s + e_i
        const long long x_lin = nbs[i];
        const int xx = (int)(x_lin % a.pitch), xy = (int)(x_lin / a.pitch);
        int nbx[9];
        int kx[9];
        links<true>(a, xx, xy, nbx, kx);
        const long long dst = ODD_NEW ? pop_loc<true>(a.plane, nbx, kx, i)
                                      : pop_loc<false>(a.plane, nbx, kx, i);
        F[dst] = F[src];
    }
    a.phi_out[s] = a.phi_out[nbz[0]];
    a.phi_out[a.plane + s] = a.phi_out[a.plane + nbz[0]];
}

}  // namespace trt
