// Two-buffer step with Phi at the current level, FP32 periodic lattices:
// persistent CTAs whose tiles (32 x 8 nodes) arrive in shared memory by TMA.
//
// Each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...; while it
// works on one tile, the tensor-memory accelerator copies the next tile's box
// (the 9 population planes of x0-4 .. x0+35 by y0-1 .. y0+8: the tile, its
// one-node halo, and the columns that keep the box's x origin on a 16-byte
// boundary) into the other of two shared-memory stages, completing on an
// mbarrier.  Phase 1 takes Phi of the tile and its halo from the stage (a
// halo cell across the lattice edge, which the box fills with zeros, is read
// at its periodic image from global memory); phase 2 collides and pushes f*
// to the other buffer as k_step_ab<S, false> does.  Every wait on an mbarrier
// is bounded: past `wait_limit` polls the CTA records the failure in *err,
// waits (bounded by TMA_WAIT_LIMIT) for its own copies in flight and returns.
#pragma once
#include <cuda.h>

#include "lb_ab.cuh"
#include "lb_ops.cuh"

namespace trt {

constexpr unsigned TMA_STAGE_BYTES = 9u * TMA_BY * TMA_BX * 4u;
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

template <typename S>
__global__ void __launch_bounds__(AB_TX * AB_TY, 4)
    k_step_ab_tma(const __grid_constant__ CUtensorMap tmap, Args<float> a, float* __restrict__ dst,
                  int tiles_x, int ntiles, int* __restrict__ err, long long wait_limit) {
    static_assert(sizeof(S) == 4, "FP32 storage only");
    __shared__ __align__(128) TmaStage stage[2];
    __shared__ float sx[AB_TY][AB_TX + 2];
    __shared__ float sy[AB_TY + 2][AB_TX];
    __shared__ __align__(8) unsigned long long bar[2];
    const float* __restrict__ F = static_cast<const float*>(a.f);
    const int tid = (int)threadIdx.x, tx = tid % AB_TX, ty = tid / AB_TX;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int tile = (int)blockIdx.x;
    if (tid == 0 && tile < ntiles) {
        mbar_expect_tx(&bar[0], TMA_STAGE_BYTES);
        tma_load_box(&stage[0], &tmap, (tile % tiles_x) * AB_TX - TMA_XOFF, (tile / tiles_x) * AB_TY - 1,
                     &bar[0]);
    }
    unsigned phase0 = 0u, phase1 = 0u;   // parity of the next completion of bar[0] / bar[1]
    for (int j = 0; tile < ntiles; ++j, tile += (int)gridDim.x) {
        const int s = j & 1;
        const int next = tile + (int)gridDim.x;
        if (tid == 0 && next < ntiles) {
            // the other stage was last read before the previous iteration's
            // closing barrier; order those reads before the async write
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bar[s ^ 1], TMA_STAGE_BYTES);
            tma_load_box(&stage[s ^ 1], &tmap, (next % tiles_x) * AB_TX - TMA_XOFF,
                         (next / tiles_x) * AB_TY - 1, &bar[s ^ 1]);
        }
        const unsigned ph = s ? phase1 : phase0;
        const bool ok = mbar_wait(&bar[s], ph, wait_limit);
        if (s) phase1 ^= 1u;
        else phase0 ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                if (err) atomicExch(err, 1);
                mbar_wait(&bar[s], ph);                                          // the late copy
                if (next < ntiles) mbar_wait(&bar[s ^ 1], s ? phase0 : phase1);   // the next one
            }
            return;
        }
        const TmaStage& st = stage[s];
        const int x0 = (tile % tiles_x) * AB_TX, y0 = (tile / tiles_x) * AB_TY;
        const int x = x0 + tx, y = y0 + ty;
        const bool inside = x < a.nx && y < a.ny;

        // phase 1: Phi of the tile and its halo
        float d[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = st.v[i][ty + 1][tx + TMA_XOFF];
        float px = 0.f, py = 0.f;
        if (inside) {
            float rho, ux, uy;
            moments_of<float>(d, a.gx, a.gy, a.rho0, rho, ux, uy);
            px = rho * ux * ux * ux;
            py = rho * uy * uy * uy;
        } else if ((x == a.nx && y < a.ny) || (y == a.ny && x < a.nx)) {
            tma_phi_global(a, F, ab_wrap(x, a.nx), ab_wrap(y, a.ny), px, py);
        }
        sx[ty][tx + 1] = px;
        sy[ty + 1][tx] = py;
        if (tid < 2 * AB_TY) {                          // left / right halo columns
            const int r = tid % AB_TY, side = tid / AB_TY;
            const int hx = side ? x0 + AB_TX : x0 - 1, hy = y0 + r;
            float qx = 0.f, qy = 0.f;
            if (hy < a.ny && (side ? x0 + AB_TX - 1 < a.nx : true)) {
                if (hx >= 0 && hx < a.nx) tma_phi_smem(a, st, hx - x0 + TMA_XOFF, r + 1, qx, qy);
                else tma_phi_global(a, F, ab_wrap(hx, a.nx), hy, qx, qy);
            }
            sx[r][side ? AB_TX + 1 : 0] = qx;
        } else if (tid < 2 * AB_TY + 2 * AB_TX) {       // bottom / top halo rows
            const int k = tid - 2 * AB_TY;
            const int c = k % AB_TX, side = k / AB_TX;
            const int hx = x0 + c, hy = side ? y0 + AB_TY : y0 - 1;
            float qx = 0.f, qy = 0.f;
            if (hx < a.nx && (side ? y0 + AB_TY - 1 < a.ny : true)) {
                if (hy >= 0 && hy < a.ny) tma_phi_smem(a, st, c + TMA_XOFF, side ? AB_TY + 1 : 0, qx, qy);
                else tma_phi_global(a, F, hx, ab_wrap(hy, a.ny), qx, qy);
            }
            sy[side ? AB_TY + 1 : 0][c] = qy;
        }
        __syncthreads();

        // phase 2: collide and push
        if (inside) {
            const float dpx = 0.5f * (sx[ty][tx + 2] - sx[ty][tx]);
            const float dpy = 0.5f * (sy[ty + 2][tx] - sy[ty][tx]);
            float o[9], phx, phy;
            collide<float>(d, dpx, dpy, a.k1, a.k1lo, a.k2, a.k2lo, a.kf, a.gx, a.gy, a.rho0, o, phx, phy);
            const int xm = ab_wrap(x - 1, a.nx), xp = ab_wrap(x + 1, a.nx);
            const long long rm = (long long)ab_wrap(y - 1, a.ny) * a.pitch;
            const long long r0 = (long long)y * a.pitch;
            const long long rp = (long long)ab_wrap(y + 1, a.ny) * a.pitch;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const long long row = ey(i) > 0 ? rp : (ey(i) < 0 ? rm : r0);
                const int col = ex(i) > 0 ? xp : (ex(i) < 0 ? xm : x);
                dst[(long long)i * a.plane + row + col] = o[i];
            }
        }
        __syncthreads();   // sx, sy and this stage are free again
    }
}

}  // namespace trt
