// Two-buffer step with Phi at the current level (G_CURRENT) for lattices
// periodic in x and y without a mask, walking down columns.
//
// The state is the canonical f(t) in buffer A, as for k_step_ab.  A warp owns
// a band of band_h rows and the 32 consecutive columns x0 - 1 .. x0 + 30,
// x0 = COL_W * (its column group): lanes 1 .. 30 update the columns x0 ..
// x0 + 29, lanes 0 and 31 stand on the two columns beside them.  Walking down
// the band, every lane loads the nine populations of its column's node in the
// next row (coalesced: 32 consecutive values of each plane), takes its moments
// and Phi = rho u^3 (eq_Gi) there, and then the inner lanes collide the node of
// the current row: d_x Phi_xxx from the two neighbouring lanes' Phi (warp
// shuffles), d_y Phi_yyy from the rows above and below, which the walk keeps
// in registers (central differences, reading R1), and the collision itself
// from the moments kept from the previous row.  f*_i goes to B[i][x + e_i]
// (periodic wrap) as in k_step_ab.  No shared memory, no barrier: a warp needs
// nothing from another warp, and the rows above and below a band, and the
// columns beside a group, are loaded again by the warps that border them
// (L2 hits; 2 of every band_h rows and 2 of every 32 columns).  Loading the
// row after next while a row collides (software pipelining) measured slower,
// into registers (they cost a quarter of the resident warps) and into a
// per-warp shared-memory ring by cp.async alike.
#pragma once
#include "lb_device.cuh"

namespace trt {

constexpr int COL_W = 30;       // columns a warp updates
constexpr int COL_WARPS = 8;    // warps per CTA

// Tallest band, in rows, for populations of elem_bytes bytes: shorter bands
// give more warps (and reload 2 rows of every band); measured on 3 x 4096^2
// (ms per step, bands of 64 / 32 / 16 rows): FP32 0.712 / 0.697 / 0.703, FP16
// 0.547 / 0.524 / 0.522, FP64 11.66 / 11.01 / 10.84.
__host__ __device__ constexpr int col_h_max(int elem_bytes) { return elem_bytes == 8 ? 16 : 32; }

// Resident CTAs per SM the column kernel asks the compiler to allow.
__host__ __device__ constexpr int col_blocks(int elem_bytes) { return elem_bytes == 8 ? 2 : 4; }
template <typename S>
__host__ __device__ constexpr int col_min_blocks() {
    return col_blocks((int)sizeof(S));
}

// Rows per band for an nx x ny lattice of elem_bytes-byte populations on a
// device of `sms` SMs: the tallest of h_max, h_max / 2 and h_max / 4 whose
// warps (one per band and group of COL_W columns) fill at least half of the
// resident warp slots; 0 when even the shortest bands leave more than half of
// them empty (the walk of a band is sequential, so few warps leave the loads'
// latency bare).  Measured on GB300 (ms per step; plain kernel / bands of
// h_max / bands of h_max / 4): FP16 1024^2 0.0162 / 0.0241 / 0.0135, 512^2
// 0.0056 / 0.0236 / 0.0076; FP64 1024^2 0.289 / 0.255 / 0.277, 512^2 0.0762 /
// 0.129 / 0.0703, 256^2 0.0231 / 0.129 / 0.0368.
inline int col_band_rows(int elem_bytes, int nx, int ny, int sms) {
    const int h_max = col_h_max(elem_bytes);
    const long long slots = (long long)sms * col_blocks(elem_bytes) * COL_WARPS;
    const long long groups = (nx + COL_W - 1) / COL_W;
    for (int h = h_max; h >= h_max / 4; h /= 2)
        if (groups * ((ny + h - 1) / h) * 2 >= slots) return h;
    return 0;
}

template <typename S>
__global__ void __launch_bounds__(COL_WARPS * 32, col_min_blocks<S>())
    k_step_ab_col(const Args<typename Fmt<S>::C> a, S* __restrict__ dst, int groups_x, int bands, int band_h) {
    using C = typename Fmt<S>::C;
    const int lane = (int)threadIdx.x & 31;
    const int gw = (int)blockIdx.x * COL_WARPS + ((int)threadIdx.x >> 5);
    if (gw >= groups_x * bands) return;   // the whole warp leaves together
    const int band = gw / groups_x;
    const int x0 = (gw - band * groups_x) * COL_W;
    const int c = x0 + lane - 1;                      // this lane's column, unwrapped
    const int cw = (c + a.nx) % a.nx;                 // ... wrapped (x0 + 30 < 2 nx + 30)
    const bool inner = lane >= 1 && lane <= COL_W && c < a.nx;
    const int y0 = band * band_h;
    const int y1 = y0 + band_h < a.ny ? y0 + band_h : a.ny;
    const S* __restrict__ F = static_cast<const S*>(a.f);
    const int xm = cw == 0 ? a.nx - 1 : cw - 1, xp = cw == a.nx - 1 ? 0 : cw + 1;

    // the moments of this lane's node in row y (wrapped)
    auto row_moments = [&](int y) {
        C d[9];
        const int k = y * a.pitch + cw;
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = Fmt<S>::ld(F[(long long)i * a.plane + k]);
        return node_moments<C>(d, a.gx, a.gy, a.rho0);
    };
    NodeMom<C> m_prev = row_moments(y0 == 0 ? a.ny - 1 : y0 - 1);
    C phy_prev = m_prev.rho * m_prev.uy * m_prev.uy * m_prev.uy;
    NodeMom<C> m_cur = row_moments(y0);
    C phx_cur = m_cur.rho * m_cur.ux * m_cur.ux * m_cur.ux;
    C phy_cur = m_cur.rho * m_cur.uy * m_cur.uy * m_cur.uy;
    for (int y = y0; y < y1; ++y) {
        const int yn = y + 1 == a.ny ? 0 : y + 1;
        const NodeMom<C> m_next = row_moments(yn);
        const C phx_next = m_next.rho * m_next.ux * m_next.ux * m_next.ux;
        const C phy_next = m_next.rho * m_next.uy * m_next.uy * m_next.uy;
        const C left = __shfl_up_sync(0xffffffffu, phx_cur, 1);
        const C right = __shfl_down_sync(0xffffffffu, phx_cur, 1);
        if (inner) {
            const C dpx = C(0.5) * (right - left);
            const C dpy = C(0.5) * (phy_next - phy_prev);
            C o[9], phx, phy;
            collide_from<C>(m_cur, dpx, dpy, a.k1, a.k1lo, a.k2, a.k2lo, a.kf, a.gx, a.gy, o, phx, phy);
            // in-plane offsets in 32 bits (a plane holds fewer than 2^31 nodes)
            const int rm = (y == 0 ? a.ny - 1 : y - 1) * a.pitch;
            const int r0 = y * a.pitch;
            const int rp = yn * a.pitch;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int row = ey(i) > 0 ? rp : (ey(i) < 0 ? rm : r0);
                const int col = ex(i) > 0 ? xp : (ex(i) < 0 ? xm : cw);
                dst[(long long)i * a.plane + row + col] = Fmt<S>::st(o[i]);
            }
        }
        phy_prev = phy_cur;
        m_cur = m_next;
        phx_cur = phx_next;
        phy_cur = phy_next;
    }
}

}  // namespace trt
