// FP64 lattice diagnostics that allocate nothing.
//
// Some callers cannot call cudaMalloc at the moment they need diagnostics: a
// host application that hands this library only memory carved from its own
// pool under a fixed device budget, or code on a latency-critical path where
// an allocation's implicit synchronisation is not acceptable.  This entry
// point serves them: the caller passes the populations, the optional mask and
// the output buffer, all in device memory it already owns, and the
// reduction's per-block partial sums go to a file-scope static device array
// that every GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "lb_device.cuh"
#include "trtrlb.h"

namespace {
constexpr int kThreads = 256;
constexpr int kNodesPerThread = 8;
constexpr int kChunk = kThreads * kNodesPerThread;  // nodes per reduction block
constexpr int kMaxBlocks = 8192;
constexpr int kValues = 8;
constexpr long long kMaxNodes = (long long)kChunk * kMaxBlocks;  // 16,777,216 (4096^2)
constexpr int kMaxDevices = 64;
}  // namespace

// Partial sums of the reduction: kValues doubles per block, 512 KiB in total.
static __device__ __align__(256) double g_diag_scratch[kMaxBlocks * kValues];

namespace {

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_diag_scratch on the current device, looked up once per
// device.  In host code the symbol is only a host-side stand-in; the kernel
// must be given the address cudaGetSymbolAddress returns.
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_diag_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

struct Canon {
    const double* f;       // [9][ny][nx]
    const uint8_t* mask;   // [ny][nx] or nullptr
    int nx, ny, px, py;
    double gx, gy;
};

// True when x + e_i is a stationary wall: a solid node, or outside a
// non-periodic edge (except the open edge of a pressure outlet node).
__device__ __forceinline__ bool wall_link(const Canon& c, int x, int y, int i, bool pressure) {
    int xn = x + trt::ex(i), yn = y + trt::ey(i);
    if (pressure && trt::ex(i) > 0) return false;
    if (xn < 0 || xn >= c.nx) {
        if (!c.px) return true;
        xn = (xn + c.nx) % c.nx;
    }
    if (yn < 0 || yn >= c.ny) {
        if (!c.py) return true;
        yn = (yn + c.ny) % c.ny;
    }
    return c.mask && c.mask[(long long)yn * c.nx + xn] == trt::SOLID;
}

// Level 1: block b reduces nodes [b * kChunk, (b + 1) * kChunk) in a fixed
// order and stores its kValues partials in scratch[b].
__global__ void __launch_bounds__(kThreads) k_diag_static_partial(Canon c, double* scratch) {
    const long long n = (long long)c.nx * c.ny;
    const long long base = (long long)blockIdx.x * kChunk;
    double acc[kValues] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int r = 0; r < kNodesPerThread; ++r) {
        const long long k = base + (long long)r * kThreads + threadIdx.x;
        if (k >= n) break;
        const int cls = c.mask ? c.mask[k] : trt::FLUID;
        if (!trt::collides(cls)) continue;
        const int x = (int)(k % c.nx), y = (int)(k / c.nx);
        double f[9];
        bool finite = true;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            f[i] = c.f[(long long)i * n + k];
            finite = finite && isfinite(f[i]);
        }
        if (!finite) {
            acc[5] += 1.0;
            continue;
        }
        double rho = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            rho += f[i];
            jx += trt::ex(i) * f[i];
            jy += trt::ey(i) * f[i];
        }
        const double ux = jx / rho + 0.5 * c.gx, uy = jy / rho + 0.5 * c.gy;
        acc[0] += rho;
        acc[1] += rho * ux;
        acc[2] += rho * uy;
        acc[3] += 0.5 * rho * (ux * ux + uy * uy);
        acc[4] = fmax(acc[4], sqrt(ux * ux + uy * uy));
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if (wall_link(c, x, y, i, cls == trt::PRESSURE)) {
                acc[6] += 2.0 * trt::ex(i) * f[trt::opp(i)];
                acc[7] += 2.0 * trt::ey(i) * f[trt::opp(i)];
            }
        }
    }
    __shared__ double sh[kValues][kThreads];
#pragma unroll
    for (int q = 0; q < kValues; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int q = 0; q < kValues; ++q) {
                const double o = sh[q][threadIdx.x + s];
                sh[q][threadIdx.x] = q == 4 ? fmax(sh[q][threadIdx.x], o) : sh[q][threadIdx.x] + o;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kValues; ++q) scratch[(long long)blockIdx.x * kValues + q] = sh[q][0];
    }
}

// Level 2: one block folds the nblocks partials in a fixed order into out.
__global__ void __launch_bounds__(kThreads) k_diag_static_final(const double* scratch, int nblocks,
                                                               double* out) {
    double acc[kValues] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads) {
#pragma unroll
        for (int q = 0; q < kValues; ++q) {
            const double v = scratch[(long long)b * kValues + q];
            acc[q] = q == 4 ? fmax(acc[q], v) : acc[q] + v;
        }
    }
    __shared__ double sh[kValues][kThreads];
#pragma unroll
    for (int q = 0; q < kValues; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int q = 0; q < kValues; ++q) {
                const double o = sh[q][threadIdx.x + s];
                sh[q][threadIdx.x] = q == 4 ? fmax(sh[q][threadIdx.x], o) : sh[q][threadIdx.x] + o;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kValues; ++q) out[q] = sh[q][0];
    }
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int trtrlb_diagnostics_noalloc(const double* f, const uint8_t* mask, int32_t nx,
                                          int32_t ny, int32_t periodic_x, int32_t periodic_y,
                                          double gx, double gy, double* out, void* stream) {
    if (nx < 1 || ny < 1) return TRTRLB_EINVAL;
    if ((long long)nx * ny > kMaxNodes) return TRTRLB_EINVAL;  // beyond the static scratch
    if (!f || !out || !is_device_pointer(f) || !is_device_pointer(out)) return TRTRLB_EINVAL;
    if (mask && !is_device_pointer(mask)) return TRTRLB_EINVAL;
    double* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return TRTRLB_ECUDA;
    }
    Canon c{f, mask, nx, ny, periodic_x ? 1 : 0, periodic_y ? 1 : 0, gx, gy};
    const long long n = (long long)nx * ny;
    const int nblocks = (int)((n + kChunk - 1) / kChunk);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_diag_static_partial<<<nblocks, kThreads, 0, st>>>(c, scratch);
    k_diag_static_final<<<1, kThreads, 0, st>>>(scratch, nblocks, out);
    return cudaGetLastError() == cudaSuccess ? TRTRLB_OK : TRTRLB_ECUDA;
}
