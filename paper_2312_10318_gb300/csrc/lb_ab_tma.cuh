// Two-buffer step with Phi at the current level, FP32 periodic lattices:
// persistent CTAs whose tiles (32 x TMA_TH nodes) arrive in shared memory by
// TMA.
//
// Each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...; while it
// works on one tile, the tensor-memory accelerator copies the boxes of the
// next TMA_STAGES - 1 tiles (the 9 population planes of x0-4 .. x0+35 by
// y0-1 .. y0+TMA_TH: the tile, its one-node halo, and the columns that keep
// the box's x origin on a 16-byte boundary) into the other shared-memory
// stages, each completing on its own mbarrier.  A thread owns the nodes of
// its column in rows ty, ty + 8, ...  Phase 1 takes Phi of the tile and its
// halo from the stage (a halo cell across the lattice edge, which the box
// fills with zeros, is read at its periodic image from global memory); phase
// 2 collides and pushes f* to the other buffer as k_step_ab<S, false> does.
// One launch may advance several lattices (TmaGroup): their tiles are
// numbered one lattice after the other and each tile finds its lattice by a
// binary search over the prefix sums.
// Every wait on an mbarrier is bounded: past `wait_limit` polls the CTA
// records the failure in the error flag of every lattice of the launch, waits
// (bounded by TMA_WAIT_LIMIT) for its own copies in flight and returns.
#pragma once
#include <cuda.h>

#include "lb_ab.cuh"
#include "lb_ops.cuh"

namespace trt {

constexpr unsigned TMA_STAGE_BYTES = 9u * TMA_BY * TMA_BX * 4u;
constexpr int TMA_R = TMA_TH / AB_TY;   // nodes per thread
static_assert(TMA_TH % AB_TY == 0 && TMA_STAGES >= 2, "tile height and stage count");
constexpr long long TMA_WAIT_LIMIT = kDefaultWaitLimit;

// One stage; padded so that both stages start on a 128-byte boundary.
struct TmaStage {
    float v[9][TMA_BY][TMA_BX];
    float pad[(128 - (9 * TMA_BY * TMA_BX * 4) % 128) % 128 / 4];
};
static_assert(sizeof(TmaStage) % 128 == 0, "stages must stay 128-byte aligned");

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the barrier to complete, at most `limit` polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity,
                                          long long limit = TMA_WAIT_LIMIT) {
    for (long long k = 0; k < limit; ++k)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_box(TmaStage* dst, const CUtensorMap* map, int x, int y,
                                             unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(0), "r"(smem_u32(bar))
        : "memory");
}

// Phi of the node at (x, y) (already wrapped) read from global memory.
__device__ __forceinline__ void tma_phi_global(const Args<float>& a, const float* F, int x, int y,
                                               float& px, float& py) {
    const long long k = (long long)y * a.pitch + x;
    float d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = F[(long long)i * a.plane + k];
    float rho, ux, uy;
    moments_of<float>(d, a.gx, a.gy, a.rho0, rho, ux, uy);
    px = rho * ux * ux * ux;
    py = rho * uy * uy * uy;
}

// Phi of box cell (column c, row r) of a stage.
__device__ __forceinline__ void tma_phi_smem(const Args<float>& a, const TmaStage& st, int c, int r,
                                             float& px, float& py) {
    float d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = st.v[i][r][c];
    float rho, ux, uy;
    moments_of<float>(d, a.gx, a.gy, a.rho0, rho, ux, uy);
    px = rho * ux * ux * ux;
    py = rho * uy * uy * uy;
}

// Shared memory of k_step_ab_tma (dynamic; its start is rounded up to 128 B).
struct TmaSmem {
    TmaStage stage[TMA_STAGES];
    float sx[TMA_TH][AB_TX + 2];     // Phi_xxx of the tile rows, with the left/right halo
    float sy[TMA_TH + 2][AB_TX];     // Phi_yyy of the tile columns, with the bottom/top halo
    unsigned long long bar[TMA_STAGES];
};
constexpr size_t TMA_SMEM_BYTES = sizeof(TmaSmem) + 128;

// The lattices of one launch (one for a single lattice, up to
// TMA_GROUP_MAX for a batch): descriptors of the buffers they read, their
// arguments, the buffers they write, their error flags, and the prefix sums of
// their tiles (tiles are numbered lattice after lattice).
constexpr int TMA_GROUP_MAX = 16;
template <int MAXL> struct TmaGroup {
    CUtensorMap map[MAXL];
    Args<float> a[MAXL];
    float* dst[MAXL];
    int* err[MAXL];
    int tile_begin[MAXL + 1];
    int tiles_x[MAXL];
    int n;
};

// Lattice of global tile `tile` (binary search over the prefix sums).
template <int MAXL>
__device__ __forceinline__ int tma_lattice(const TmaGroup<MAXL>& p, int tile) {
    if constexpr (MAXL == 1) return 0;   // a single lattice: its arguments at fixed offsets
    int lo = 0, hi = p.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.tile_begin[mid] <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int MAXL>
__device__ __forceinline__ void tma_issue(TmaSmem& sm, int k, const TmaGroup<MAXL>& p, int tile) {
    const int l = tma_lattice(p, tile), t = tile - p.tile_begin[l], tw = p.tiles_x[l];
    mbar_expect_tx(&sm.bar[k], TMA_STAGE_BYTES);
    tma_load_box(&sm.stage[k], &p.map[l], (t % tw) * AB_TX - TMA_XOFF, (t / tw) * TMA_TH - 1, &sm.bar[k]);
}

// Five resident CTAs per SM (at most 48 registers): the kernel is bound by
// per-tile latency, and its rate follows the resident warps (4 CTAs per SM
// measured 0.8 of the rate of 5).
template <int MAXL>
__global__ void __launch_bounds__(AB_TX * AB_TY, TMA_R == 1 ? 5 : 3)
    k_step_ab_tma(const __grid_constant__ TmaGroup<MAXL> p, int ntiles, long long wait_limit) {
    extern __shared__ unsigned char tma_smem_raw[];
    TmaSmem& sm = *reinterpret_cast<TmaSmem*>(tma_smem_raw + ((128u - (smem_u32(tma_smem_raw) & 127u)) & 127u));
    const int tid = (int)threadIdx.x, tx = tid % AB_TX, ty = tid / AB_TX;
    const int grid = (int)gridDim.x;

    if (tid == 0) {
        for (int k = 0; k < TMA_STAGES; ++k) mbar_init(&sm.bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int tile = (int)blockIdx.x;
    if (tid == 0)
        for (int k = 0; k < TMA_STAGES - 1; ++k)
            if (tile + k * grid < ntiles) tma_issue(sm, k, p, tile + k * grid);
    unsigned phases = 0u;   // bit k: parity of the next completion of bar[k]
    for (int s = 0; tile < ntiles; tile += grid, s = s + 1 == TMA_STAGES ? 0 : s + 1) {
        const int ahead = tile + (TMA_STAGES - 1) * grid;
        const int sa = s == 0 ? TMA_STAGES - 1 : s - 1;   // stage of the tile `ahead`
        if (tid == 0 && ahead < ntiles) {
            // stage sa was last read before the previous iteration's closing
            // barrier; order those reads before the async write
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_issue(sm, sa, p, ahead);
        }
        const unsigned ph = (phases >> s) & 1u;
        const bool ok = mbar_wait(&sm.bar[s], ph, wait_limit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                for (int k = 0; k < p.n; ++k)   // the tiles this CTA leaves are lost
                    if (p.err[k]) atomicExch(p.err[k], 1);
                // the copies in flight: this tile's and those of the next
                // TMA_STAGES - 1 tiles
                for (int k = 0; k < TMA_STAGES; ++k) {
                    const int sk = (s + k) % TMA_STAGES;
                    if (tile + k * grid < ntiles) mbar_wait(&sm.bar[sk], (phases >> sk) & 1u);
                }
            }
            return;
        }
        phases ^= 1u << s;
        const TmaStage& st = sm.stage[s];
        const int lat = tma_lattice(p, tile);
        const Args<float>& a = p.a[lat];
        const float* __restrict__ F = static_cast<const float*>(a.f);
        float* __restrict__ dst = p.dst[lat];
        const int lt = tile - p.tile_begin[lat], tiles_x = p.tiles_x[lat];
        const int x0 = (lt % tiles_x) * AB_TX, y0 = (lt / tiles_x) * TMA_TH;
        const int x = x0 + tx;

        // phase 1: Phi of the tile and its halo; the tile nodes keep their
        // moments for the collision
        NodeMom<float> m[TMA_R];
#pragma unroll
        for (int r = 0; r < TMA_R; ++r) {
            const int ry = ty + r * AB_TY, y = y0 + ry;
            float d[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) d[i] = st.v[i][ry + 1][tx + TMA_XOFF];
            m[r] = node_moments<float>(d, a.gx, a.gy, a.rho0);
            float px = 0.f, py = 0.f;
            if (x < a.nx && y < a.ny) {
                px = m[r].rho * m[r].ux * m[r].ux * m[r].ux;
                py = m[r].rho * m[r].uy * m[r].uy * m[r].uy;
            } else if ((x == a.nx && y < a.ny) || (y == a.ny && x < a.nx)) {
                tma_phi_global(a, F, ab_wrap(x, a.nx), ab_wrap(y, a.ny), px, py);
            }
            sm.sx[ry][tx + 1] = px;
            sm.sy[ry + 1][tx] = py;
        }
        if (tid < 2 * TMA_TH) {                          // left / right halo columns
            const int r = tid % TMA_TH, side = tid / TMA_TH;
            const int hx = side ? x0 + AB_TX : x0 - 1, hy = y0 + r;
            float qx = 0.f, qy = 0.f;
            if (hy < a.ny && (side ? x0 + AB_TX - 1 < a.nx : true)) {
                if (hx >= 0 && hx < a.nx) tma_phi_smem(a, st, hx - x0 + TMA_XOFF, r + 1, qx, qy);
                else tma_phi_global(a, F, ab_wrap(hx, a.nx), hy, qx, qy);
            }
            sm.sx[r][side ? AB_TX + 1 : 0] = qx;
        } else if (tid < 2 * TMA_TH + 2 * AB_TX) {       // bottom / top halo rows
            const int k = tid - 2 * TMA_TH;
            const int c = k % AB_TX, side = k / AB_TX;
            const int hx = x0 + c, hy = side ? y0 + TMA_TH : y0 - 1;
            float qx = 0.f, qy = 0.f;
            if (hx < a.nx && (side ? y0 + TMA_TH - 1 < a.ny : true)) {
                if (hy >= 0 && hy < a.ny) tma_phi_smem(a, st, c + TMA_XOFF, side ? TMA_TH + 1 : 0, qx, qy);
                else tma_phi_global(a, F, hx, ab_wrap(hy, a.ny), qx, qy);
            }
            sm.sy[side ? TMA_TH + 1 : 0][c] = qy;
        }
        __syncthreads();

        // phase 2: collide and push
        const int xm = ab_wrap(x - 1, a.nx), xp = ab_wrap(x + 1, a.nx);
#pragma unroll
        for (int r = 0; r < TMA_R; ++r) {
            const int ry = ty + r * AB_TY, y = y0 + ry;
            if (x < a.nx && y < a.ny) {
                const float dpx = 0.5f * (sm.sx[ry][tx + 2] - sm.sx[ry][tx]);
                const float dpy = 0.5f * (sm.sy[ry + 2][tx] - sm.sy[ry][tx]);
                float o[9], phx, phy;
                collide_from<float>(m[r], dpx, dpy, a.k1, a.k1lo, a.k2, a.k2lo, a.kf, a.gx, a.gy, o, phx,
                                    phy);
                // in-plane offsets in 32 bits (a plane holds fewer than 2^31 nodes)
                const int rm = ab_wrap(y - 1, a.ny) * a.pitch;
                const int r0 = y * a.pitch;
                const int rp = ab_wrap(y + 1, a.ny) * a.pitch;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const int row = ey(i) > 0 ? rp : (ey(i) < 0 ? rm : r0);
                    const int col = ex(i) > 0 ? xp : (ex(i) < 0 ? xm : x);
                    float* __restrict__ q = dst + (long long)i * a.plane;
                    q[row + col] = o[i];
                }
            }
        }
        __syncthreads();   // sx, sy and this stage are free again
    }
}

}  // namespace trt
