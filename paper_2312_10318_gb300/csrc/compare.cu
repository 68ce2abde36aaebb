// FP64 comparison of two velocity fields on the device: the relative L2 error
// of eq_n1, the largest local change of eq_n2 and the relative L2 error of the
// vorticity, by a deterministic two-level reduction (fixed node ranges per
// block, fixed tree order: the same fields always reduce to the same bits).
//
// Vorticity is omega = d_x u_y - d_y u_x by second-order central differences
// on the node lattice, at fluid nodes whose four axis neighbours are fluid
// nodes of the domain (wrapped across periodic edges); other fluid nodes enter
// the velocity sums only.
#include <cuda_runtime.h>

#include "lb_device.cuh"
#include "lb_ops.cuh"

namespace trt {

namespace {

constexpr int CMP_THREADS = 256;
constexpr int CMP_VALUES = 8;

struct CmpArgs {
    const double* ux;     // [ny][nx]
    const double* uy;
    const double* rx;     // reference, [ny][nx]
    const double* ry;
    const uint8_t* mask;  // [ny][pitch] or nullptr
    int nx, ny, pitch, px, py;
};

// Index of a neighbour along one axis, -1 outside a non-periodic edge.
__device__ __forceinline__ int wrap1(int v, int n, int periodic) {
    if (v < 0) return periodic ? v + n : -1;
    if (v >= n) return periodic ? v - n : -1;
    return v;
}

__device__ __forceinline__ bool fluid_at(const CmpArgs& a, int x, int y) {
    return !a.mask || collides(a.mask[(long long)y * a.pitch + x]);
}

// Partial sums of one block: [0] sum |du|^2, [1] sum |u_ref|^2, [2] max |du|,
// [3] sum (d omega)^2, [4] sum omega_ref^2, [5] fluid nodes, [6] nodes with a
// vorticity, [7] fluid nodes where u or u_ref is not finite.
__global__ void __launch_bounds__(CMP_THREADS) k_compare_partial(CmpArgs a, double* __restrict__ part) {
    double acc[CMP_VALUES] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long n = (long long)a.nx * a.ny;
    for (long long k = (long long)blockIdx.x * CMP_THREADS + threadIdx.x; k < n;
         k += (long long)gridDim.x * CMP_THREADS) {
        const int x = (int)(k % a.nx), y = (int)(k / a.nx);
        if (!fluid_at(a, x, y)) continue;
        const double ux = a.ux[k], uy = a.uy[k], rx = a.rx[k], ry = a.ry[k];
        if (!(isfinite(ux) && isfinite(uy) && isfinite(rx) && isfinite(ry))) {
            acc[7] += 1.0;
            continue;
        }
        const double dx = ux - rx, dy = uy - ry;
        const double d2 = dx * dx + dy * dy;
        acc[0] += d2;
        acc[1] += rx * rx + ry * ry;
        acc[2] = fmax(acc[2], sqrt(d2));
        acc[5] += 1.0;
        const int xm = wrap1(x - 1, a.nx, a.px), xp = wrap1(x + 1, a.nx, a.px);
        const int ym = wrap1(y - 1, a.ny, a.py), yp = wrap1(y + 1, a.ny, a.py);
        if (xm < 0 || xp < 0 || ym < 0 || yp < 0) continue;
        if (!fluid_at(a, xm, y) || !fluid_at(a, xp, y) || !fluid_at(a, x, ym) || !fluid_at(a, x, yp)) continue;
        const long long kxm = (long long)y * a.nx + xm, kxp = (long long)y * a.nx + xp;
        const long long kym = (long long)ym * a.nx + x, kyp = (long long)yp * a.nx + x;
        const double w = 0.5 * (a.uy[kxp] - a.uy[kxm]) - 0.5 * (a.ux[kyp] - a.ux[kym]);
        const double wr = 0.5 * (a.ry[kxp] - a.ry[kxm]) - 0.5 * (a.rx[kyp] - a.rx[kym]);
        const double dw = w - wr;
        if (!(isfinite(w) && isfinite(wr))) continue;
        acc[3] += dw * dw;
        acc[4] += wr * wr;
        acc[6] += 1.0;
    }
    __shared__ double sh[CMP_VALUES][CMP_THREADS];
#pragma unroll
    for (int q = 0; q < CMP_VALUES; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = CMP_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int q = 0; q < CMP_VALUES; ++q) {
                const double o = sh[q][threadIdx.x + s];
                sh[q][threadIdx.x] = q == 2 ? fmax(sh[q][threadIdx.x], o) : sh[q][threadIdx.x] + o;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < CMP_VALUES; ++q) part[(long long)blockIdx.x * CMP_VALUES + q] = sh[q][0];
    }
}

// num / den under a square root; 0 when both vanish, +inf for num > 0 = den.
__device__ __forceinline__ double rel_root(double num, double den) {
    if (den > 0.0) return sqrt(num / den);
    return num > 0.0 ? __longlong_as_double(0x7ff0000000000000ll) : 0.0;
}

// Folds the partials in a fixed order and writes the TRTRLB_CMP_* outputs.
__global__ void __launch_bounds__(CMP_THREADS) k_compare_final(const double* __restrict__ part, int nblocks,
                                                              double* out) {
    double acc[CMP_VALUES] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += CMP_THREADS) {
#pragma unroll
        for (int q = 0; q < CMP_VALUES; ++q) {
            const double v = part[(long long)b * CMP_VALUES + q];
            acc[q] = q == 2 ? fmax(acc[q], v) : acc[q] + v;
        }
    }
    __shared__ double sh[CMP_VALUES][CMP_THREADS];
#pragma unroll
    for (int q = 0; q < CMP_VALUES; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = CMP_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int q = 0; q < CMP_VALUES; ++q) {
                const double o = sh[q][threadIdx.x + s];
                sh[q][threadIdx.x] = q == 2 ? fmax(sh[q][threadIdx.x], o) : sh[q][threadIdx.x] + o;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double s_du = sh[0][0], s_ref = sh[1][0], n = sh[5][0];
        out[0] = rel_root(s_du, s_ref);                 // eq_n1 relative L2 of u
        out[1] = sh[2][0];                              // max |u - u_ref| (eq_n2)
        out[2] = rel_root(sh[3][0], sh[4][0]);          // relative L2 of omega
        out[3] = n > 0.0 ? sqrt(s_du / n) : 0.0;        // RMS |u - u_ref|
        out[4] = s_du;
        out[5] = s_ref;
        out[6] = sh[3][0];
        out[7] = sh[4][0];
        out[8] = n;
        out[9] = sh[7][0];
    }
}

}  // namespace

int compare_blocks(long long nodes) {
    const long long b = (nodes + CMP_THREADS - 1) / CMP_THREADS;
    return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

cudaError_t compare_fields(const double* ux, const double* uy, const double* rx, const double* ry,
                           const uint8_t* mask, int nx, int ny, int pitch, int px, int py,
                           double* part, double* out, cudaStream_t st) {
    const CmpArgs a{ux, uy, rx, ry, mask, nx, ny, pitch, px, py};
    const int nb = compare_blocks((long long)nx * ny);
    k_compare_partial<<<nb, CMP_THREADS, 0, st>>>(a, part);
    k_compare_final<<<1, CMP_THREADS, 0, st>>>(part, nb, out);
    return cudaGetLastError();
}

}  // namespace trt
