// Two-buffer step with Phi at the current time level (G_CURRENT).
//
// The state is the canonical f(t) in buffer A (F[i][x] = f_i(x, t), the same
// form as an even AA level).  A CTA owns a 32 x 8 tile.  Phase 1: every node
// of the tile and of its one-node halo (left/right columns for d_x Phi_xxx,
// top/bottom rows for d_y Phi_yyy) computes Phi = rho u^3 of the current level
// from its own populations into shared memory (walls, inlets, ghosts and the
// outside of non-periodic edges take the values of the wall reading).  Phase
// 2: each fluid node takes d Phi by central differences, collides (eq2) and
// pushes f*_i to B[i][x + e_i] (half-way bounce-back into B[ibar][x] at walls,
// with the moving-wall correction at inlets).  The inward neighbour z of an
// outlet ghost s also emits, on the ghost's behalf, f*_i(z) into every fluid
// node s + e_i.  No Phi buffers are read or written: 72 B/node in FP32, at
// twice the population memory of the in-place kernels.
#pragma once
#include "lb_device.cuh"

namespace trt {

constexpr int AB_TX = 32, AB_TY = 8;

// Class of (x, y) with wrap; OUT for outside a non-periodic edge.
enum : int { AB_OUT = 255 };

template <typename C>
__device__ __forceinline__ int ab_class(const Args<C>& a, int& x, int& y) {
    if (x < 0 || x >= a.nx) {
        if (!a.px) return AB_OUT;
        x = x < 0 ? x + a.nx : x - a.nx;
    }
    if (y < 0 || y >= a.ny) {
        if (!a.py) return AB_OUT;
        y = y < 0 ? y + a.ny : y - a.ny;
    }
    return a.mask ? a.mask[(long long)y * a.pitch + x] : FLUID;
}

// Phi_xxx, Phi_yyy of node (x, y) of the canonical state (wall reading R2;
// beyond a pressure outlet node the outlet's own value).
template <typename S>
__device__ __forceinline__ void ab_phi(const Args<typename Fmt<S>::C>& a, const S* F, int x, int y,
                                       typename Fmt<S>::C& px, typename Fmt<S>::C& py) {
    using C = typename Fmt<S>::C;
    const int x_in = x;
    int c = ab_class(a, x, y);
    if (c == AB_OUT && x_in == a.nx && y >= 0 && y < a.ny && a.mask &&
        a.mask[(long long)y * a.pitch + a.nx - 1] == PRESSURE) {
        x = a.nx - 1;
        c = PRESSURE;
    }
    if (c == AB_OUT || c == SOLID) {
        px = py = C(0);
        return;
    }
    if (c == INLET) {   // rho_w u_w^3
        px = a.phin_x;
        py = a.phin_y;
        return;
    }
    if (c == OUTLET) {   // the inward neighbour's value
        x = x == 0 ? a.nx - 1 : x - 1;
    }
    const long long k = (long long)y * a.pitch + x;
    C d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = Fmt<S>::ld(F[(long long)i * a.plane + k]);
    if (c == PRESSURE || c == HALO_PRESSURE) zh_fill<C>(d, a.zh_dr);
    C rho, ux, uy;
    moments_of<C>(d, a.gx, a.gy, a.rho0, rho, ux, uy);
    px = rho * ux * ux * ux;
    py = rho * uy * uy * uy;
}

__device__ __forceinline__ int ab_wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// GENERAL: walls, masks or non-periodic edges; otherwise the lattice is
// periodic in x and y without a mask and every link streams.
template <typename S, bool GENERAL>
__global__ void __launch_bounds__(AB_TX * AB_TY, 4) k_step_ab(Args<typename Fmt<S>::C> a, S* dst,
                                                              int g_off) {
    using C = typename Fmt<S>::C;
    __shared__ C sx[AB_TY][AB_TX + 2];   // Phi_xxx with left/right halo
    __shared__ C sy[AB_TY + 2][AB_TX];   // Phi_yyy with top/bottom halo
    const S* __restrict__ F = static_cast<const S*>(a.f);
    const int tx = (int)threadIdx.x % AB_TX, ty = (int)threadIdx.x / AB_TX;
    const int x0 = blockIdx.x * AB_TX, y0 = blockIdx.y * AB_TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool inside = x < a.nx && y < a.ny;

    const long long own = (long long)y * a.pitch + x;
    const int cls = (GENERAL && a.mask && inside) ? a.mask[own] : FLUID;
    const bool fluid = inside && collides(cls);
    C d[9];
    if (fluid) {
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = Fmt<S>::ld(F[(long long)i * a.plane + own]);
        if (GENERAL && cls == PRESSURE) zh_fill<C>(d, a.zh_dr);
    }

    // phase 1: Phi of the tile and its halo.  A shared cell holds Phi of its
    // (wrapped) position only if some lattice node of the tile reads it: the
    // tile's own nodes, the column x = nx and row y = ny just past a partial
    // tile's edge (the periodic neighbours of the last column and row), and
    // the halo column/row next to a full tile edge.  Every position computed is
    // within one node of the lattice, so one wrap brings it inside.
    if (!g_off && !GENERAL) {
        // periodic lattice: every thread loads its halo node (if it has one)
        // together with its own node, so the two load latencies overlap
        const int h = (int)threadIdx.x;
        int hx = -1, hy = -1;                     // wrapped halo position
        if (h < 2 * AB_TY) {                      // left / right halo columns
            const int r = h % AB_TY, side = h / AB_TY;
            if (y0 + r < a.ny && (side ? x0 + AB_TX - 1 < a.nx : true)) {
                hx = ab_wrap(side ? x0 + AB_TX : x0 - 1, a.nx);
                hy = y0 + r;
            }
        } else if (h < 2 * AB_TY + 2 * AB_TX) {   // bottom / top halo rows
            const int k = h - 2 * AB_TY;
            const int c = k % AB_TX, side = k / AB_TX;
            if (x0 + c < a.nx && (side ? y0 + AB_TY - 1 < a.ny : true)) {
                hx = x0 + c;
                hy = ab_wrap(side ? y0 + AB_TY : y0 - 1, a.ny);
            }
        }
        // the cell just past a partial tile's last column / row
        const bool past = !inside && ((x == a.nx && y < a.ny) || (y == a.ny && x < a.nx));
        C e[9];
        if (past) {
            const long long k = (long long)ab_wrap(y, a.ny) * a.pitch + ab_wrap(x, a.nx);
#pragma unroll
            for (int i = 0; i < 9; ++i) d[i] = Fmt<S>::ld(F[(long long)i * a.plane + k]);
        }
        if (hx >= 0) {
            const long long k = (long long)hy * a.pitch + hx;
#pragma unroll
            for (int i = 0; i < 9; ++i) e[i] = Fmt<S>::ld(F[(long long)i * a.plane + k]);
        }
        C px = C(0), py = C(0);
        if (inside || past) {
            C rho, ux, uy;
            moments_of<C>(d, a.gx, a.gy, a.rho0, rho, ux, uy);
            px = rho * ux * ux * ux;
            py = rho * uy * uy * uy;
        }
        sx[ty][tx + 1] = px;
        sy[ty + 1][tx] = py;
        if (h < 2 * AB_TY + 2 * AB_TX) {
            C qx = C(0), qy = C(0);
            if (hx >= 0) {
                C rho, ux, uy;
                moments_of<C>(e, a.gx, a.gy, a.rho0, rho, ux, uy);
                qx = rho * ux * ux * ux;
                qy = rho * uy * uy * uy;
            }
            if (h < 2 * AB_TY) sx[h % AB_TY][h / AB_TY ? AB_TX + 1 : 0] = qx;
            else sy[(h - 2 * AB_TY) / AB_TX ? AB_TY + 1 : 0][(h - 2 * AB_TY) % AB_TX] = qy;
        }
        __syncthreads();
    } else if (!g_off) {
        C px = C(0), py = C(0);
        if (fluid) {
            C rho, ux, uy;
            moments_of<C>(d, a.gx, a.gy, a.rho0, rho, ux, uy);
            px = rho * ux * ux * ux;
            py = rho * uy * uy * uy;
        } else if (inside || (x == a.nx && y < a.ny) || (y == a.ny && x < a.nx)) {
            ab_phi<S>(a, F, x, y, px, py);
        }
        sx[ty][tx + 1] = px;
        sy[ty + 1][tx] = py;
        const int h = (int)threadIdx.x;
        if (h < 2 * AB_TY) {                       // left / right halo columns
            const int hy = h % AB_TY, side = h / AB_TY;
            const int hx = side ? x0 + AB_TX : x0 - 1;
            C qx = C(0), qy = C(0);
            const bool needed = y0 + hy < a.ny && (side ? x0 + AB_TX - 1 < a.nx : true);
            if (needed) ab_phi<S>(a, F, hx, y0 + hy, qx, qy);
            sx[hy][side ? AB_TX + 1 : 0] = qx;
        } else if (h < 2 * AB_TY + 2 * AB_TX) {    // bottom / top halo rows
            const int k = h - 2 * AB_TY;
            const int hx = k % AB_TX, side = k / AB_TX;
            const int hy = side ? y0 + AB_TY : y0 - 1;
            C qx = C(0), qy = C(0);
            const bool needed = x0 + hx < a.nx && (side ? y0 + AB_TY - 1 < a.ny : true);
            if (needed) ab_phi<S>(a, F, x0 + hx, hy, qx, qy);
            sy[side ? AB_TY + 1 : 0][hx] = qy;
        }
        __syncthreads();
    }
    if (!fluid) return;

    // phase 2: collide the node and push
    C dpx = C(0), dpy = C(0);
    if (!g_off) {
        // the halo outside a non-periodic edge holds 0 (stationary wall)
        dpx = C(0.5) * (sx[ty][tx + 2] - sx[ty][tx]);
        dpy = C(0.5) * (sy[ty + 2][tx] - sy[ty][tx]);
    }
    C o[9], phx, phy;
    collide<C>(d, dpx, dpy, a.k1, a.k1lo, a.k2, a.k2lo, a.kf, a.gx, a.gy, a.rho0, o, phx, phy);
    if (!GENERAL) {
        const int xm = ab_wrap(x - 1, a.nx), xp = ab_wrap(x + 1, a.nx);
        const long long rm = (long long)ab_wrap(y - 1, a.ny) * a.pitch;
        const long long r0 = (long long)y * a.pitch;
        const long long rp = (long long)ab_wrap(y + 1, a.ny) * a.pitch;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const long long row = ey(i) > 0 ? rp : (ey(i) < 0 ? rm : r0);
            const int col = ex(i) > 0 ? xp : (ex(i) < 0 ? xm : x);
            dst[(long long)i * a.plane + row + col] = Fmt<S>::st(o[i]);
        }
        return;
    }
    // is (x, y) the inward neighbour of an outlet ghost?
    int gx = x + 1, gy = y;
    const bool proxy = a.mask && ab_class(a, gx, gy) == OUTLET;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int txn = x + ex(i), tyn = y + ey(i);
        const int c = i == 0 ? FLUID : ab_class(a, txn, tyn);
        if (collides(c) || c == HALO || c == HALO_PRESSURE) {
            dst[(long long)i * a.plane + (long long)tyn * a.pitch + txn] = Fmt<S>::st(o[i]);
        } else if (c == SOLID || c == AB_OUT) {
            // (across the edge of a pressure outlet this fills a population
            // that the Zou-He rebuild replaces when it is read)
            dst[(long long)opp(i) * a.plane + own] = Fmt<S>::st(o[i]);
        } else if (c == INLET) {
            dst[(long long)opp(i) * a.plane + own] = Fmt<S>::st(o[i] - a.corr[i]);
        }
        // links into an outlet ghost are dropped
        if (proxy && i != 0) {
            int sxn = gx + ex(i), syn = gy + ey(i);
            if (collides(ab_class(a, sxn, syn)))
                dst[(long long)i * a.plane + (long long)syn * a.pitch + sxn] = Fmt<S>::st(o[i]);
        }
    }
}

}  // namespace trt
