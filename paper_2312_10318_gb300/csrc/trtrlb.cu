// C ABI of the D2Q9 TRT-RLB library (declared in include/trtrlb.h).
// Owns the device memory of each lattice, validates the problem statement and
// dispatches to the per-format launchers (lb_ops.cuh).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lb_ab_col.cuh"
#include "lb_handle.h"


namespace {

thread_local char g_create_err[256] = "";

// Device doubles of a handle's result buffer (diagnostics: 8, comparisons:
// TRTRLB_CMP_N).
constexpr int kResultDoubles = 16;
static_assert(TRTRLB_CMP_N <= kResultDoubles, "comparison results exceed the result buffer");

size_t elem_size(int storage) {
    switch (storage) {
        case TRTRLB_F64: return sizeof(double);
        case TRTRLB_F64_DW: return sizeof(double);
        case TRTRLB_F32: return sizeof(float);
        case TRTRLB_F16_SHIFTED: return sizeof(__half);
        case TRTRLB_BF16_SHIFTED: return sizeof(__nv_bfloat16);
        default: return 0;
    }
}
size_t phi_size(int storage) {
    return (storage == TRTRLB_F64 || storage == TRTRLB_F64_DW) ? 8 : sizeof(float);
}

int fail(char* buf, int code, const char* fmt, const char* detail = nullptr) {
    if (detail) std::snprintf(buf, 256, fmt, detail);
    else std::snprintf(buf, 256, "%s", fmt);
    return code;
}

int cuda_fail(char* buf, cudaError_t e, const char* where) {
    std::snprintf(buf, 256, "%s: %s", where, cudaGetErrorString(e));
    return TRTRLB_ECUDA;
}

bool on_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Dispatch of Ops<S> on the storage format.
#define TRT_DISPATCH(storage, CALL)                                              \
    [&]() -> cudaError_t {                                                       \
        switch (storage) {                                                       \
            case TRTRLB_F64: { using S = double; return trt::Ops<S>::CALL; }     \
            case TRTRLB_F64_DW: { using S = trt::f64dw; return trt::Ops<S>::CALL; } \
            case TRTRLB_F32: { using S = float; return trt::Ops<S>::CALL; }      \
            case TRTRLB_F16_SHIFTED: { using S = __half; return trt::Ops<S>::CALL; } \
            default: { using S = __nv_bfloat16; return trt::Ops<S>::CALL; }      \
        }                                                                        \
    }()

void release(trtrlb_lattice* h) {
    if (!h) return;
    if (h->f) cudaFree(h->f);
    if (h->f2) cudaFree(h->f2);
    if (h->phi) cudaFree(h->phi);
    if (h->mask) cudaFree(h->mask);
    if (h->ghosts) cudaFree(h->ghosts);
    if (h->seg) cudaFree(h->seg);
    if (h->stage) cudaFree(h->stage);
    if (h->part) cudaFree(h->part);
    if (h->dout) cudaFree(h->dout);
    if (h->kerr) cudaFree(h->kerr);
    delete[] static_cast<CUtensorMap*>(h->tmaps);
    delete h;
}

// TRTRLB_ETIMEOUT if a kernel of the handle reported a bounded wait that ran
// out (the flag is cleared); call after the handle's stream is synchronised.
int check_kerr(trtrlb_lattice* h) {
    if (!h->kerr) return TRTRLB_OK;
    int v = 0;
    if (cudaMemcpy(&v, h->kerr, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return TRTRLB_ECUDA;
    if (!v) return TRTRLB_OK;
    cudaMemsetAsync(h->kerr, 0, sizeof v, h->stream);
    return fail(h->err, TRTRLB_ETIMEOUT, "a step kernel's wait for its tile copy ran out");
}

// The vector kernel needs a periodic lattice without mask and nx divisible
// by its width.
bool vector_applies(const trtrlb_lattice* h) {
    return !h->s.general && h->p.g_mode != TRTRLB_G_CURRENT &&
           h->p.nx % trt::vec_width((int)elem_size(h->p.storage)) == 0;
}

// Default kernel: the vector kernel for the 32- and 16-bit formats (measured
// faster on GB300), the scalar one for the 64-bit formats (as fast for FP64,
// faster for double-word storage, whose pairs double the vector kernel's
// registers).  The autotuner may choose otherwise.
bool auto_vector(const trtrlb_lattice* h) {
    const int st = h->p.storage;
    return vector_applies(h) && st != TRTRLB_F64 && st != TRTRLB_F64_DW;
}

// Default two-buffer kernel of a G_CURRENT lattice that is periodic without a
// mask: for FP64, FP16 and BF16 storage the column-walking kernel wherever its
// bands give enough warps (trt::col_band_rows; on 3 x 4096^2 it stepped FP16
// in 0.551 ms against 0.696 for the plain kernel, FP64 in 11.66 against
// 13.75), the plain kernel below that; FP32 keeps the TMA-fed kernel, which
// measured faster from 2048^2 (one 4096^2 lattice: 0.2297 against 0.2306 ms).
// Returns the column kernel's rows per band, 0 when it is not the default.
int auto_column(const trtrlb_lattice* h) {
    const int st = h->p.storage;
    if (h->p.g_mode != TRTRLB_G_CURRENT || h->s.general ||
        !(st == TRTRLB_F64 || st == TRTRLB_F16_SHIFTED || st == TRTRLB_BF16_SHIFTED))
        return 0;
    return trt::col_band_rows((int)elem_size(st), h->p.nx, h->p.ny, h->sms);
}

// Row segments of 32 nodes (x = 32 s .. 32 s + 31 of row y) whose nodes are
// plain fluid nodes, and so is each of their eight neighbours, inside the
// domain or across a periodic edge: walls, mask classes and open edges touch
// none of their links, so the general step runs the periodic step's code
// there.  A 3 x 3 erosion of the fluid set, then an AND per segment.
std::vector<uint8_t> interior_segments(const uint8_t* mask, int nx, int ny, bool px, bool py) {
    const int segs = (nx + 31) / 32;
    std::vector<uint8_t> fl((size_t)nx * ny), hx((size_t)nx * ny), seg((size_t)ny * segs, 0);
    for (size_t k = 0; k < fl.size(); ++k) fl[k] = !mask || mask[k] == TRTRLB_FLUID;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t r = (size_t)y * nx;
            const bool l = x > 0 ? fl[r + x - 1] : (px && fl[r + nx - 1]);
            const bool rr = x < nx - 1 ? fl[r + x + 1] : (px && fl[r]);
            hx[r + x] = fl[r + x] && l && rr;
        }
    for (int y = 0; y < ny; ++y) {
        const int ym = y > 0 ? y - 1 : (py ? ny - 1 : -1), yp = y < ny - 1 ? y + 1 : (py ? 0 : -1);
        for (int sgi = 0; sgi < segs; ++sgi) {
            bool ok = ym >= 0 && yp >= 0;
            const int x1 = sgi * 32 + 32 < nx ? sgi * 32 + 32 : nx;
            for (int x = sgi * 32; ok && x < x1; ++x)
                ok = hx[(size_t)y * nx + x] && hx[(size_t)ym * nx + x] && hx[(size_t)yp * nx + x];
            seg[(size_t)y * segs + sgi] = ok ? 1 : 0;
        }
    }
    return seg;
}

// Staging buffer for host transfers and comparisons: at least `fields` FP64
// fields of nx * ny values, allocated on first use and grown when a call needs
// more (3 for moments and init, 4 for comparisons, 11 for populations and
// Phi).  Growing frees the old buffer, which waits for the work queued on it.
cudaError_t ensure_stage(trtrlb_lattice* h, int fields) {
    const size_t n = (size_t)h->p.nx * h->p.ny;
    if (h->stage && h->stage_fields >= fields) return cudaSuccess;
    if (h->stage) {
        cudaFree(h->stage);
        h->bytes -= (int64_t)(sizeof(double) * h->stage_fields * n);
        h->stage = nullptr;
        h->stage_fields = 0;
    }
    const size_t bytes = sizeof(double) * fields * n;
    const cudaError_t e = cudaMalloc((void**)&h->stage, bytes);
    if (e == cudaSuccess) {
        h->bytes += (int64_t)bytes;
        h->stage_fields = fields;
    } else {
        h->stage = nullptr;
    }
    return e;
}

// TMA descriptor of one FP32 population buffer for k_step_ab_tma: a 3-D tensor
// (x: nx, y: ny rows of `pitch` floats, plane: 9 planes of ny * pitch floats)
// read in boxes of 40 x (TMA_TH + 2) x 9 (the 32 x TMA_TH tile, its one-node
// halo and the columns that keep the box origin 16-byte aligned); outside the
// lattice the box is filled with zeros.
cudaError_t encode_tma(void* base, int nx, int ny, int pitch, CUtensorMap* out) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                                               cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !ptr) return cudaErrorNotSupported;
        fn = reinterpret_cast<Encode>(ptr);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 9};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)trt::TMA_BX, (cuuint32_t)trt::TMA_BY, 9};
    const cuuint32_t elem[3] = {1, 1, 1};
    const CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, elem,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Resolves tau_s2 from tau_s2 / magic (eq_a29).  Returns 0 or an error code.
int resolve_tau2(const trtrlb_params& p, double* tau2, char* err) {
    const bool has_t2 = !std::isnan(p.tau_s2), has_m = !std::isnan(p.magic);
    if (!has_t2 && !has_m) return fail(err, TRTRLB_EINVAL, "one of tau_s2 / magic must be given");
    double t2 = has_t2 ? p.tau_s2 : 0.5 + p.magic / (p.tau_s - 0.5);
    if (has_t2 && has_m) {
        const double from_m = 0.5 + p.magic / (p.tau_s - 0.5);
        if (std::fabs(from_m - t2) > 1e-12 * std::fabs(t2))
            return fail(err, TRTRLB_EINVAL, "tau_s2 and magic disagree");
    }
    // tau_s2 = 1/2 (1/tau_s2 = 2, the end of the stability sweep of Sec. III A)
    // mirrors the third-order non-equilibrium; below it the factor exceeds 1
    if (!(t2 >= 0.5) || !std::isfinite(t2))
        return fail(err, TRTRLB_EINVAL, "tau_s2 must be finite and >= 1/2 (magic >= 0)");
    *tau2 = t2;
    return 0;
}

}  // namespace

extern "C" {

void trtrlb_default_params(trtrlb_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->nx = p->ny = 64;
    p->periodic_x = p->periodic_y = 1;
    p->tau_s = 0.8;
    p->tau_s2 = NAN;
    p->magic = 0.25;
    p->rho0 = 1.0;
    p->wall_rho = 1.0;
    p->outlet_rho = 1.0;
    p->storage = TRTRLB_F32;
    p->g_mode = TRTRLB_G_LAGGED;
}

int trtrlb_create(const trtrlb_params* pp, const uint8_t* mask, void* stream, trtrlb_t* out) {
    char* err = g_create_err;
    err[0] = 0;
    if (!pp || !out) return fail(err, TRTRLB_EINVAL, "null params or output handle");
    const trtrlb_params p = *pp;
    // grid rows are launched as gridDim.y = ceil(ny / 8) <= 65535; node offsets
    // (including padding) fit in 32-bit integers
    if (p.nx < 1 || p.ny < 1 || p.ny > 131070 || p.nx > (1 << 24) ||
        ((int64_t)p.nx + 63) * p.ny > (int64_t)1 << 30)
        return fail(err, TRTRLB_EINVAL, "lattice size out of range");
    if (!(p.tau_s > 0.5) || !std::isfinite(p.tau_s))
        return fail(err, TRTRLB_EINVAL, "tau_s must be finite and > 1/2");
    double tau2 = 0;
    if (int rc = resolve_tau2(p, &tau2, err)) return rc;
    if (elem_size(p.storage) == 0) return fail(err, TRTRLB_EINVAL, "unknown storage format");
    if (p.g_mode != TRTRLB_G_LAGGED && p.g_mode != TRTRLB_G_OFF && p.g_mode != TRTRLB_G_CURRENT)
        return fail(err, TRTRLB_EINVAL, "unknown g_mode");
    if (!(p.rho0 > 0) || !std::isfinite(p.gx) || !std::isfinite(p.gy) ||
        !std::isfinite(p.wall_ux) || !std::isfinite(p.wall_uy) || !std::isfinite(p.wall_rho))
        return fail(err, TRTRLB_EINVAL, "rho0 must be > 0 and forces / wall state finite");
    if (!(p.outlet_rho > 0) || !std::isfinite(p.outlet_rho))
        return fail(err, TRTRLB_EINVAL, "outlet_rho must be finite and > 0");

    const int pitch = (p.nx + 63) / 64 * 64;
    const long long plane = (long long)pitch * p.ny;
    std::vector<int> ghosts;
    if (mask) {
        for (int y = 0; y < p.ny; ++y)
            for (int x = 0; x < p.nx; ++x) {
                const uint8_t c = mask[(long long)y * p.nx + x];
                if (c > TRTRLB_HALO_PRESSURE) return fail(err, TRTRLB_EINVAL, "mask class out of range");
                if (c == TRTRLB_PRESSURE && (p.periodic_x || x != p.nx - 1))
                    return fail(err, TRTRLB_EINVAL,
                                "pressure outlet nodes must lie on the last column of a lattice not periodic in x");
                if (c != TRTRLB_OUTLET) continue;
                int zx = x - 1;
                if (zx < 0) {
                    if (!p.periodic_x) return fail(err, TRTRLB_EINVAL, "outlet ghost without inward neighbour");
                    zx += p.nx;
                }
                if (mask[(long long)y * p.nx + zx] != TRTRLB_FLUID)
                    return fail(err, TRTRLB_EINVAL, "outlet ghost's inward neighbour (x-1,y) must be fluid");
                // the inward neighbour's links toward -x must not end at a moving wall
                for (int dy = -1; dy <= 1; ++dy) {
                    int qx = zx - 1, qy = y + dy;
                    if (qx < 0) { if (!p.periodic_x) continue; qx += p.nx; }
                    if (qy < 0 || qy >= p.ny) { if (!p.periodic_y) continue; qy = (qy + p.ny) % p.ny; }
                    if (mask[(long long)qy * p.nx + qx] == TRTRLB_INLET)
                        return fail(err, TRTRLB_EINVAL, "outlet ghost too close to an inlet");
                }
                ghosts.push_back((int)((long long)y * pitch + x));
            }
    }

    trtrlb_lattice* h = new (std::nothrow) trtrlb_lattice();
    if (!h) return fail(err, TRTRLB_ENOMEM, "host allocation failed");
    h->p = p;
    h->p.tau_s2 = tau2;
    h->p.magic = (p.tau_s - 0.5) * (tau2 - 0.5);
    h->stream = static_cast<cudaStream_t>(stream);
    const size_t es = elem_size(p.storage), ps = phi_size(p.storage);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(err, e, "device query");
    }
    auto alloc = [&](void** ptr, size_t bytes) {
        e = cudaMalloc(ptr, bytes);
        if (e == cudaSuccess) h->bytes += (int64_t)bytes;
        return e == cudaSuccess;
    };
    bool ok = alloc(&h->f, es * 9 * plane) && alloc(&h->phi, ps * 4 * plane) &&
              alloc((void**)&h->dout, sizeof(double) * kResultDoubles);
    if (ok && p.g_mode == TRTRLB_G_CURRENT) ok = alloc(&h->f2, es * 9 * plane);
    if (ok && mask) ok = alloc((void**)&h->mask, (size_t)plane);
    if (ok && !ghosts.empty()) ok = alloc((void**)&h->ghosts, sizeof(int) * ghosts.size());
    trt::State& s = h->s;
    s.f = h->f;
    s.f2 = h->f2;
    s.phi[0] = h->phi;
    s.phi[1] = static_cast<char*>(h->phi) + ps * 2 * plane;
    s.cur = 0;
    s.mask = h->mask;
    s.ghosts = h->ghosts;
    s.nghost = (int)ghosts.size();
    s.nx = p.nx; s.ny = p.ny; s.pitch = pitch; s.plane = plane;
    s.px = p.periodic_x ? 1 : 0; s.py = p.periodic_y ? 1 : 0;
    s.general = mask != nullptr || !p.periodic_x || !p.periodic_y;
    s.g_mode = p.g_mode;
    s.tau1 = p.tau_s; s.tau2 = tau2;
    s.gx = p.gx; s.gy = p.gy; s.rho0 = p.rho0;
    s.wall_ux = p.wall_ux; s.wall_uy = p.wall_uy; s.wall_rho = p.wall_rho;
    s.outlet_rho = p.outlet_rho;
    s.parity = 0;
    s.wait_limit = trt::kDefaultWaitLimit;
    if (ok) ok = alloc((void**)&h->part, sizeof(double) * 8 * trt::diag_blocks(s));
    if (!ok) {
        const int rc = e == cudaErrorMemoryAllocation ? TRTRLB_ENOMEM : TRTRLB_ECUDA;
        std::snprintf(err, 256, "cudaMalloc: %s", cudaGetErrorString(e));
        cudaGetLastError();
        release(h);
        return rc;
    }
    if (mask) {
        // pitched copy of the mask; padding columns are marked solid
        std::vector<uint8_t> m((size_t)plane, TRTRLB_SOLID);
        for (int y = 0; y < p.ny; ++y)
            std::memcpy(&m[(size_t)y * pitch], mask + (size_t)y * p.nx, p.nx);
        e = cudaMemcpy(h->mask, m.data(), (size_t)plane, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !ghosts.empty())
            e = cudaMemcpy(h->ghosts, ghosts.data(), sizeof(int) * ghosts.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            const int rc = cuda_fail(err, e, "mask upload");
            release(h);
            return rc;
        }
    }
    if (s.general) {
        const std::vector<uint8_t> seg = interior_segments(mask, p.nx, p.ny, p.periodic_x, p.periodic_y);
        e = cudaMalloc((void**)&h->seg, seg.size());
        if (e == cudaSuccess) {
            h->bytes += (int64_t)seg.size();
            e = cudaMemcpy(h->seg, seg.data(), seg.size(), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            const int rc = cuda_fail(err, e, "segment map");
            release(h);
            return rc;
        }
        s.seg = h->seg;
        s.segs = (p.nx + 31) / 32;
    }
    e = cudaMemsetAsync(h->f, 0, es * 9 * plane, h->stream);
    if (e == cudaSuccess && h->f2) e = cudaMemsetAsync(h->f2, 0, es * 9 * plane, h->stream);
    if (e == cudaSuccess) e = TRT_DISPATCH(p.storage, phi_static(h->s, h->stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        const int rc = cuda_fail(err, e, "create");
        release(h);
        return rc;
    }
    h->t = 0;
    h->tile_w = p.nx >= 128 ? 128 : (p.nx >= 64 ? 64 : 32);
    s.tile_w = h->tile_w;
    h->variant = TRTRLB_KERNEL_AUTO;
    s.vec = auto_vector(h);
    s.col_h = auto_column(h);
    if (p.g_mode == TRTRLB_G_CURRENT && p.storage == TRTRLB_F32 && !s.general) {
        // the TMA-fed two-buffer kernel; without a descriptor the plain one runs
        CUtensorMap* maps = new (std::nothrow) CUtensorMap[2];
        e = maps ? cudaMalloc((void**)&h->kerr, sizeof(int)) : cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaMemsetAsync(h->kerr, 0, sizeof(int), h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess) e = encode_tma(h->f, p.nx, p.ny, pitch, &maps[0]);
        if (e == cudaSuccess) e = encode_tma(h->f2, p.nx, p.ny, pitch, &maps[1]);
        if (e == cudaSuccess) {
            h->tmaps = maps;
            s.tma_buf[0] = h->f;
            s.tma_buf[1] = h->f2;
            s.tma_map[0] = &maps[0];
            s.tma_map[1] = &maps[1];
            s.kerr = h->kerr;
            h->tma_grid = trt::Ops<float>::tma_grid();
            s.tma_grid = h->tma_grid;
        } else {
            delete[] maps;
            if (h->kerr) cudaFree(h->kerr);
            h->kerr = nullptr;
            cudaGetLastError();
        }
    }
    *out = h;
    return TRTRLB_OK;
}

int trtrlb_destroy(trtrlb_t h) {
    if (!h) return TRTRLB_OK;
    cudaStreamSynchronize(h->stream);
    release(h);
    return TRTRLB_OK;
}

int trtrlb_set_stream(trtrlb_t h, void* stream) {
    if (!h) return TRTRLB_EINVAL;
    h->stream = static_cast<cudaStream_t>(stream);
    return TRTRLB_OK;
}

int trtrlb_init(trtrlb_t h, const double* rho, const double* ux, const double* uy) {
    if (!h) return TRTRLB_EINVAL;
    h->err[0] = 0;
    if (!ux || !uy) return fail(h->err, TRTRLB_EINVAL, "ux and uy are required");
    const size_t n = (size_t)h->p.nx * h->p.ny, nb = n * sizeof(double);
    const double* src[3] = {rho, ux, uy};
    const double* dev[3] = {nullptr, nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 3 && e == cudaSuccess; ++q) {
        if (!src[q]) continue;
        if (on_device(src[q])) {
            dev[q] = src[q];
        } else {
            e = ensure_stage(h, 3);
            if (e != cudaSuccess) break;
            e = cudaMemcpyAsync(h->stage + q * n, src[q], nb, cudaMemcpyHostToDevice, h->stream);
            dev[q] = h->stage + q * n;
        }
    }
    if (e == cudaSuccess) e = TRT_DISPATCH(h->p.storage, init(h->s, dev[0], dev[1], dev[2], h->stream));
    if (e != cudaSuccess) return cuda_fail(h->err, e, "init");
    h->t = 0;
    return TRTRLB_OK;
}

int trtrlb_step(trtrlb_t h, int64_t nsteps) {
    if (!h) return TRTRLB_EINVAL;
    h->err[0] = 0;
    if (nsteps < 0) return fail(h->err, TRTRLB_EINVAL, "nsteps must be >= 0");
    for (int64_t k = 0; k < nsteps; ++k) {
        const cudaError_t e = TRT_DISPATCH(h->p.storage, step(h->s, h->stream));
        if (e != cudaSuccess) return cuda_fail(h->err, e, "step");
        ++h->t;
    }
    return TRTRLB_OK;
}

int trtrlb_moments(trtrlb_t h, double* rho, double* ux, double* uy) {
    if (!h) return TRTRLB_EINVAL;
    h->err[0] = 0;
    const size_t n = (size_t)h->p.nx * h->p.ny, nb = n * sizeof(double);
    double* dst[3] = {rho, ux, uy};
    double* dev[3] = {nullptr, nullptr, nullptr};
    bool host = false;
    for (int q = 0; q < 3; ++q)
        if (dst[q] && !on_device(dst[q])) host = true;
    if (host) {
        const cudaError_t se = ensure_stage(h, 3);
        if (se != cudaSuccess) return cuda_fail(h->err, se, "moments staging");
    }
    for (int q = 0; q < 3; ++q) {
        if (!dst[q]) continue;
        dev[q] = on_device(dst[q]) ? dst[q] : h->stage + q * n;
    }
    cudaError_t e = TRT_DISPATCH(h->p.storage, moments(h->s, dev[0], dev[1], dev[2], h->stream));
    for (int q = 0; q < 3 && e == cudaSuccess; ++q)
        if (dst[q] && dev[q] != dst[q])
            e = cudaMemcpyAsync(dst[q], dev[q], nb, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && host) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h->err, e, "moments");
    return host ? check_kerr(h) : TRTRLB_OK;
}

int trtrlb_get_f(trtrlb_t h, double* f, double* phi) {
    if (!h) return TRTRLB_EINVAL;
    h->err[0] = 0;
    const size_t n = (size_t)h->p.nx * h->p.ny;
    if ((f && !on_device(f)) || (phi && !on_device(phi))) {
        const cudaError_t se = ensure_stage(h, 11);
        if (se != cudaSuccess) return cuda_fail(h->err, se, "get_f staging");
    }
    double* df = f && !on_device(f) ? h->stage : f;
    double* dp = phi && !on_device(phi) ? h->stage + 9 * n : phi;
    cudaError_t e = TRT_DISPATCH(h->p.storage, get_f(h->s, df, dp, h->stream));
    bool host = false;
    if (e == cudaSuccess && f && df != f) {
        e = cudaMemcpyAsync(f, df, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        host = true;
    }
    if (e == cudaSuccess && phi && dp != phi) {
        e = cudaMemcpyAsync(phi, dp, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        host = true;
    }
    if (e == cudaSuccess && host) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h->err, e, "get_f");
    return host ? check_kerr(h) : TRTRLB_OK;
}

// ---- checkpoint image -------------------------------------------------------
namespace {

struct ImageHeader {
    uint64_t magic;                   // "TRTRLBS1"
    int32_t nx, ny, storage, g_mode;
    int32_t parity, cur, pitch, reserved;
    int64_t t;
};
constexpr uint64_t kImageMagic = 0x3153424c52545254ull;   // bytes "TRTRLBS1"

size_t image_pop_bytes(const trtrlb_lattice* h) { return elem_size(h->p.storage) * 9 * (size_t)h->s.plane; }
size_t image_phi_bytes(const trtrlb_lattice* h) { return phi_size(h->p.storage) * 4 * (size_t)h->s.plane; }

}  // namespace

int64_t trtrlb_state_bytes(trtrlb_t h) {
    if (!h) return -1;
    return (int64_t)(sizeof(ImageHeader) + image_pop_bytes(h) + image_phi_bytes(h));
}

int trtrlb_save(trtrlb_t h, void* image) {
    if (!h || !image) return TRTRLB_EINVAL;
    h->err[0] = 0;
    ImageHeader hd{kImageMagic, h->p.nx, h->p.ny, h->p.storage, h->p.g_mode,
                   h->s.parity, h->s.cur, h->s.pitch, 0, h->t};
    char* out = static_cast<char*>(image);
    cudaError_t e = cudaMemcpyAsync(out, &hd, sizeof hd, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out + sizeof hd, h->s.f, image_pop_bytes(h), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out + sizeof hd + image_pop_bytes(h), h->phi, image_phi_bytes(h),
                            cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h->err, e, "save");
    return TRTRLB_OK;
}

int trtrlb_load(trtrlb_t h, const void* image) {
    if (!h || !image) return TRTRLB_EINVAL;
    h->err[0] = 0;
    const char* in = static_cast<const char*>(image);
    ImageHeader hd;
    cudaError_t e = cudaMemcpy(&hd, in, sizeof hd, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(h->err, e, "load");
    if (hd.magic != kImageMagic || hd.nx != h->p.nx || hd.ny != h->p.ny || hd.storage != h->p.storage ||
        hd.g_mode != h->p.g_mode || hd.pitch != h->s.pitch || (hd.parity & ~1) || (hd.cur & ~1))
        return fail(h->err, TRTRLB_EINVAL, "state image does not match this lattice");
    e = cudaMemcpyAsync(h->s.f, in + sizeof hd, image_pop_bytes(h), cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->phi, in + sizeof hd + image_pop_bytes(h), image_phi_bytes(h),
                            cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h->err, e, "load");
    h->s.parity = hd.parity;
    h->s.cur = hd.cur;
    h->t = hd.t;
    return TRTRLB_OK;
}

int trtrlb_set_f(trtrlb_t h, const double* f, const double* phi) {
    if (!h) return TRTRLB_EINVAL;
    h->err[0] = 0;
    if (!f) return fail(h->err, TRTRLB_EINVAL, "f is required");
    const size_t n = (size_t)h->p.nx * h->p.ny;
    const double* df = f;
    const double* dp = phi;
    cudaError_t e = cudaSuccess;
    if (!on_device(f) || (phi && !on_device(phi))) e = ensure_stage(h, 11);
    if (e == cudaSuccess && !on_device(f)) {
        e = cudaMemcpyAsync(h->stage, f, 9 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        df = h->stage;
    }
    if (e == cudaSuccess && phi && !on_device(phi)) {
        e = cudaMemcpyAsync(h->stage + 9 * n, phi, 2 * n * sizeof(double), cudaMemcpyHostToDevice,
                            h->stream);
        dp = h->stage + 9 * n;
    }
    if (e == cudaSuccess) e = TRT_DISPATCH(h->p.storage, set_f(h->s, df, dp, h->stream));
    if (e != cudaSuccess) return cuda_fail(h->err, e, "set_f");
    h->t = 0;
    return TRTRLB_OK;
}

int64_t trtrlb_time(trtrlb_t h) { return h ? h->t : -1; }

int trtrlb_diagnostics(trtrlb_t h, double* out) {
    if (!h || !out) return TRTRLB_EINVAL;
    h->err[0] = 0;
    const bool dev = on_device(out);
    cudaError_t e = TRT_DISPATCH(h->p.storage, diagnostics(h->s, h->part, dev ? out : h->dout, h->stream));
    if (e == cudaSuccess && !dev) {
        e = cudaMemcpyAsync(out, h->dout, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h->err, e, "diagnostics");
    return dev ? TRTRLB_OK : check_kerr(h);
}

}  // extern "C"

namespace {

// u of h (eq11) into ux, uy (dense FP64 device fields) on `stream`.
cudaError_t velocity_into(trtrlb_lattice* h, double* ux, double* uy, cudaStream_t stream) {
    return TRT_DISPATCH(h->p.storage, moments(h->s, nullptr, ux, uy, stream));
}

// Comparison of a's velocity (in a's staging buffer) with rx, ry (device), into
// out (host or device).
int compare_into(trtrlb_lattice* a, const double* rx, const double* ry, double* out, bool host_out) {
    const size_t n = (size_t)a->p.nx * a->p.ny;
    cudaError_t e = trt::compare_fields(a->stage, a->stage + n, rx, ry, a->mask, a->p.nx, a->p.ny,
                                        a->s.pitch, a->s.px, a->s.py, a->part, host_out ? a->dout : out,
                                        a->stream);
    if (e == cudaSuccess && host_out) {
        e = cudaMemcpyAsync(out, a->dout, TRTRLB_CMP_N * sizeof(double), cudaMemcpyDeviceToHost,
                            a->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(a->stream);
    }
    if (e != cudaSuccess) return cuda_fail(a->err, e, "compare");
    return host_out ? check_kerr(a) : TRTRLB_OK;
}

}  // namespace

extern "C" {

int trtrlb_compare(trtrlb_t h, const double* ux_ref, const double* uy_ref, double* out) {
    if (!h) return TRTRLB_EINVAL;
    h->err[0] = 0;
    if (!ux_ref || !uy_ref || !out) return fail(h->err, TRTRLB_EINVAL, "ux_ref, uy_ref and out are required");
    const size_t n = (size_t)h->p.nx * h->p.ny;
    cudaError_t e = ensure_stage(h, 4);
    if (e != cudaSuccess) return cuda_fail(h->err, e, "compare staging");
    const double* ref[2] = {ux_ref, uy_ref};
    const double* dev[2];
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
        if (on_device(ref[q])) {
            dev[q] = ref[q];
        } else {
            e = cudaMemcpyAsync(h->stage + (2 + q) * n, ref[q], n * sizeof(double), cudaMemcpyHostToDevice,
                                h->stream);
            dev[q] = h->stage + (2 + q) * n;
        }
    }
    if (e == cudaSuccess) e = velocity_into(h, h->stage, h->stage + n, h->stream);
    if (e != cudaSuccess) return cuda_fail(h->err, e, "compare");
    return compare_into(h, dev[0], dev[1], out, !on_device(out));
}

int trtrlb_compare_lattices(trtrlb_t a, trtrlb_t b, double* out) {
    if (!a || !b) return TRTRLB_EINVAL;
    a->err[0] = 0;
    if (!out) return fail(a->err, TRTRLB_EINVAL, "out is required");
    if (a->p.nx != b->p.nx || a->p.ny != b->p.ny) return fail(a->err, TRTRLB_EINVAL, "lattice sizes differ");
    const size_t n = (size_t)a->p.nx * a->p.ny;
    cudaError_t e = ensure_stage(a, 4);
    if (e != cudaSuccess) return cuda_fail(a->err, e, "compare staging");
    // b's queued work before the read of its state on a's stream, and b's
    // later work after it
    cudaEvent_t ev = nullptr;
    const bool other = a->stream != b->stream;
    if (other) {
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(a->stream, ev, 0);
    }
    if (e == cudaSuccess) e = velocity_into(b, a->stage + 2 * n, a->stage + 3 * n, a->stream);
    if (e == cudaSuccess) e = velocity_into(a, a->stage, a->stage + n, a->stream);
    if (e == cudaSuccess && other) e = cudaEventRecord(ev, a->stream);
    if (e == cudaSuccess && other) e = cudaStreamWaitEvent(b->stream, ev, 0);
    if (ev) cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_fail(a->err, e, "compare");
    return compare_into(a, a->stage + 2 * n, a->stage + 3 * n, out, !on_device(out));
}

}  // extern "C"

extern "C" {

int64_t trtrlb_device_bytes(trtrlb_t h) { return h ? h->bytes : -1; }

int trtrlb_set_kernel(trtrlb_t h, int32_t variant, int32_t tile_w) {
    if (!h) return TRTRLB_EINVAL;
    h->err[0] = 0;
    if (tile_w != 0 && tile_w != 32 && tile_w != 64 && tile_w != 128 && tile_w != 256)
        return fail(h->err, TRTRLB_EINVAL, "tile_w must be 0, 32, 64, 128 or 256");
    const bool can_vec = vector_applies(h);
    bool vec;
    switch (variant) {
        case TRTRLB_KERNEL_AUTO: vec = auto_vector(h); break;
        case TRTRLB_KERNEL_SCALAR: vec = false; break;
        case TRTRLB_KERNEL_VECTOR:
            if (!can_vec)
                return fail(h->err, TRTRLB_ENOTSUP,
                            "the vector kernel needs a periodic lattice without mask and nx divisible by its width");
            vec = true;
            break;
        case TRTRLB_KERNEL_COLUMN:
            if (h->p.g_mode != TRTRLB_G_CURRENT || h->s.general || h->p.storage == TRTRLB_F64_DW)
                return fail(h->err, TRTRLB_ENOTSUP,
                            "the column kernel needs G_CURRENT, a periodic lattice without mask and FP64, FP32, FP16 or BF16 storage");
            vec = false;
            break;
        default: return fail(h->err, TRTRLB_EINVAL, "unknown kernel variant");
    }
    h->variant = variant;
    h->s.vec = vec;
    if (variant == TRTRLB_KERNEL_COLUMN) {
        // the tallest band that still fills the device, else the shortest
        const int es = (int)elem_size(h->p.storage);
        const int band = trt::col_band_rows(es, h->p.nx, h->p.ny, h->sms);
        h->s.col_h = band > 0 ? band : trt::col_h_max(es) / 4;
    } else {
        h->s.col_h = variant == TRTRLB_KERNEL_AUTO ? auto_column(h) : 0;
    }
    // G_CURRENT: AUTO runs the TMA-fed kernel where it exists, SCALAR the plain
    // one, COLUMN the column-walking one
    h->s.tma_grid = variant == TRTRLB_KERNEL_AUTO || variant == TRTRLB_KERNEL_VECTOR ? h->tma_grid : 0;
    if (tile_w) h->tile_w = h->s.tile_w = tile_w;
    return TRTRLB_OK;
}

int trtrlb_set_wait_limit(trtrlb_t h, int64_t polls) {
    if (!h) return TRTRLB_EINVAL;
    h->err[0] = 0;
    if (polls < 0) return fail(h->err, TRTRLB_EINVAL, "polls must be >= 0");
    h->s.wait_limit = polls;
    return TRTRLB_OK;
}

int trtrlb_get_kernel(trtrlb_t h, int32_t* vector, int32_t* tile_w) {
    if (!h) return TRTRLB_EINVAL;
    if (vector) *vector = h->s.vec ? 1 : 0;
    if (tile_w) *tile_w = h->tile_w;
    return TRTRLB_OK;
}

int trtrlb_step_kernel(trtrlb_t h, int32_t* kind) {
    if (!h || !kind) return TRTRLB_EINVAL;
    if (h->p.g_mode != TRTRLB_G_CURRENT)
        *kind = h->s.vec ? TRTRLB_STEP_AA_VECTOR : TRTRLB_STEP_AA;
    else if (h->p.storage == TRTRLB_F32 && trt::Ops<float>::tma_eligible(h->s))
        *kind = shares_tma_launch(h) ? TRTRLB_STEP_AB_TMA_SHARED : TRTRLB_STEP_AB_TMA;
    else if (h->s.col_h > 0 && !h->s.general && h->p.storage != TRTRLB_F64_DW)
        *kind = TRTRLB_STEP_AB_COLUMN;
    else
        *kind = TRTRLB_STEP_AB;
    return TRTRLB_OK;
}

const char* trtrlb_strerror(int code) {
    switch (code) {
        case TRTRLB_OK: return "ok";
        case TRTRLB_EINVAL: return "invalid argument";
        case TRTRLB_ENOMEM: return "out of memory";
        case TRTRLB_ECUDA: return "CUDA error";
        case TRTRLB_EUNSTABLE: return "unstable state (NaN/Inf or velocity bound exceeded)";
        case TRTRLB_ETIMEOUT: return "bounded wait timed out";
        case TRTRLB_ENOTSUP: return "not supported";
        default: return "unknown error";
    }
}

const char* trtrlb_last_error(trtrlb_t h) { return h ? h->err : g_create_err; }

}  // extern "C"

namespace trt {

// a[k], or null when the array itself is null
template <typename T>
static T* at(T* const* a, int k) {
    return a ? a[k] : nullptr;
}

// End-to-end solve of several lattices with the copies beside the steps (the
// body of trtrlb_batch_solve): uploads on `cin`, member k's steps on `st`, its
// initial state and moments on `aux` (beside the neighbouring members' steps),
// its downloads on `cout` once its moments are written.
int solve_members(trtrlb_lattice* const* m, int count, cudaStream_t st, cudaStream_t aux, cudaStream_t cin,
                  cudaStream_t cout, const double* const* rho, const double* const* ux, const double* const* uy,
                  int64_t nsteps, double* const* rho_out, double* const* ux_out, double* const* uy_out,
                  char* err) {
    if (count < 0 || (count > 0 && (!m || !ux || !uy)) || nsteps < 0)
        return fail(err, TRTRLB_EINVAL, "bad member list, input arrays or step count");
    for (int k = 0; k < count; ++k)
        if (!m[k] || !ux[k] || !uy[k]) return fail(err, TRTRLB_EINVAL, "every member needs ux and uy");
    if (count == 0) return TRTRLB_OK;
    // events per member: uploaded, initialised, stepped, moments written; and one
    // for the members' earlier work
    std::vector<cudaEvent_t> ev(4 * (size_t)count + 1, nullptr);
    cudaEvent_t* ev_in = ev.data();
    cudaEvent_t* ev_init = ev.data() + count;
    cudaEvent_t* ev_step = ev.data() + 2 * count;
    cudaEvent_t* ev_mom = ev.data() + 3 * count;
    cudaEvent_t ev_prior = ev[4 * (size_t)count];
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    ev_prior = ev[4 * (size_t)count];
    // staging for host inputs and outputs (allocated before any copy is queued)
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        const void* io[6] = {at(rho, k), ux[k], uy[k], at(rho_out, k), at(ux_out, k), at(uy_out, k)};
        bool host = false;
        for (const void* p : io) host = host || (p && !on_device(p));
        if (host) e = ensure_stage(m[k], 3);
    }
    // every member's earlier work (on its own stream) before this call's
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        e = cudaEventRecord(ev_prior, m[k]->stream);
        for (cudaStream_t x : {st, aux, cin, cout})
            if (e == cudaSuccess) e = cudaStreamWaitEvent(x, ev_prior, 0);
    }
    std::vector<const double*> din(3 * (size_t)count, nullptr);
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        const size_t n = (size_t)m[k]->p.nx * m[k]->p.ny;
        const double* src[3] = {at(rho, k), ux[k], uy[k]};
        for (int q = 0; q < 3 && e == cudaSuccess; ++q) {
            if (!src[q] || on_device(src[q])) {
                din[3 * k + q] = src[q];
                continue;
            }
            e = cudaMemcpyAsync(m[k]->stage + q * n, src[q], n * sizeof(double), cudaMemcpyHostToDevice, cin);
            din[3 * k + q] = m[k]->stage + q * n;
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_in[k], cin);
    }
    // initial states on the auxiliary stream, each as soon as its fields are up
    // (member k + 1's beside member k's steps)
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        trtrlb_lattice* h = m[k];
        e = cudaStreamWaitEvent(aux, ev_in[k], 0);
        if (e == cudaSuccess)
            e = TRT_DISPATCH(h->p.storage, init(h->s, din[3 * k], din[3 * k + 1], din[3 * k + 2], aux));
        if (e == cudaSuccess) e = cudaEventRecord(ev_init[k], aux);
        h->t = 0;
    }
    // the steps, member after member; each member's moments on the auxiliary
    // stream and its download on the copy stream, beside the next member's steps
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        trtrlb_lattice* h = m[k];
        const size_t n = (size_t)h->p.nx * h->p.ny;
        e = cudaStreamWaitEvent(st, ev_init[k], 0);
        for (int64_t q = 0; q < nsteps && e == cudaSuccess; ++q) {
            e = TRT_DISPATCH(h->p.storage, step(h->s, st));
            ++h->t;
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_step[k], st);
        double* dst[3] = {at(rho_out, k), at(ux_out, k), at(uy_out, k)};
        double* dev[3] = {nullptr, nullptr, nullptr};
        for (int q = 0; q < 3; ++q)
            if (dst[q]) dev[q] = on_device(dst[q]) ? dst[q] : h->stage + q * n;
        if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, ev_step[k], 0);
        if (e == cudaSuccess && (dev[0] || dev[1] || dev[2]))
            e = TRT_DISPATCH(h->p.storage, moments(h->s, dev[0], dev[1], dev[2], aux));
        if (e == cudaSuccess) e = cudaEventRecord(ev_mom[k], aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cout, ev_mom[k], 0);
        for (int q = 0; q < 3 && e == cudaSuccess; ++q)
            if (dst[q] && dev[q] != dst[q])
                e = cudaMemcpyAsync(dst[q], dev[q], n * sizeof(double), cudaMemcpyDeviceToHost, cout);
    }
    cudaError_t es = cudaSuccess;
    for (cudaStream_t x : {cout, st, aux, cin}) {
        const cudaError_t ex_ = cudaStreamSynchronize(x);
        if (es == cudaSuccess) es = ex_;
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) return cuda_fail(err, e, "solve");
    for (int k = 0; k < count; ++k)
        if (const int rc = check_kerr(m[k])) {
            std::snprintf(err, 256, "%s", m[k]->err);
            return rc;
        }
    return TRTRLB_OK;
}

int diag_blocks(const State& s) {
    const long long n = (long long)s.nx * s.ny;
    long long b = (n + DIAG_THREADS - 1) / DIAG_THREADS;
    return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}
}  // namespace trt
