// Batched step: one launch advances a group of lattices that share storage
// format, boundary flavour, G mode and the parity of their current level.  The
// lattices' arguments travel in the kernel's parameter space (constant bank),
// so a CTA finds its lattice and reads its coefficients with uniform constant
// loads; the per-node body is the fully specialised node_step.
#pragma once
#include "lb_device.cuh"
#include "lb_vec.cuh"

namespace trt {

constexpr int BATCH_THREADS = 256;

template <typename C, int MAXL> struct GroupParams {
    int n;                       // lattices in this launch
    int tile_begin[MAXL + 1];    // prefix sums of tiles; tile_begin[n] = total
    int tiles_x[MAXL];           // tiles per tile row
    int log2_tw[MAXL];           // scalar: tile width 2^log2_tw nodes, height 256 / width
    int segs[MAXL];              // vector: warp segments per row
    float inv_d[MAXL];           // 1 / tiles_x (scalar) or 1 / segs (vector), rounded
    Args<C> a[MAXL];
};

// q = t / d and r = t % d for 0 <= t < 2^24 and d >= 1, from the rounded
// reciprocal inv = 1/d: the float estimate of t/d is within 2^-23 relative,
// so its truncation is off by at most one, which one compare corrects.
__device__ __forceinline__ void tile_divmod(int t, int d, float inv, int& q, int& r) {
    q = __float2int_rz(__fmul_rn((float)t, inv));
    r = t - q * d;
    if (r < 0) {
        --q;
        r += d;
    } else if (r >= d) {
        ++q;
        r -= d;
    }
}

template <typename S, bool ODD, bool GENERAL, int GMODE, int MAXL>
__global__ void __launch_bounds__(BATCH_THREADS, step_min_blocks<S, GENERAL, GMODE>())
    k_step_group(const __grid_constant__ GroupParams<typename Fmt<S>::C, MAXL> p) {
    const int b = (int)blockIdx.x;
    int lo = 0, hi = p.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.tile_begin[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const int lt = p.log2_tw[lo];
    const int t = b - p.tile_begin[lo];
    int tx, ty;
    tile_divmod(t, p.tiles_x[lo], p.inv_d[lo], ty, tx);
    const int x = (tx << lt) + ((int)threadIdx.x & ((1 << lt) - 1));
    const int y = (ty << (8 - lt)) + ((int)threadIdx.x >> lt);
    if (x >= p.a[lo].nx || y >= p.a[lo].ny) return;
    node_step<S, ODD, GENERAL, GMODE>(p.a[lo], x, y);
}

// Vectorised flavour: a CTA owns 8 consecutive warp segments of one lattice.
template <typename S, bool ODD, int GMODE, int MAXL>
__global__ void __launch_bounds__(BATCH_THREADS, sizeof(S) == 2 ? 4 : 3)
    k_step_group_vec(const __grid_constant__ GroupParams<typename Fmt<S>::C, MAXL> p) {
    constexpr int V = Pk<S>::V;
    const int b = (int)blockIdx.x;
    int lo = 0, hi = p.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.tile_begin[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const int lane = (int)threadIdx.x & 31;
    const int s = (b - p.tile_begin[lo]) * 8 + ((int)threadIdx.x >> 5);   // < 2^24
    const int spr = p.segs[lo];
    if ((long long)s >= (long long)spr * p.a[lo].ny) return;   // whole warp leaves together
    int y, sx;
    tile_divmod(s, spr, p.inv_d[lo], y, sx);
    const int x0 = sx * 32 * V + lane * V;
    seg_step<S, ODD, GMODE>(p.a[lo], x0, y, lane);
}

}  // namespace trt
