// Slab decomposition: one lattice split into sub-lattices of consecutive rows,
// each a lattice handle of its own with halo rows (class TRTRLB_HALO) facing
// its neighbours, and a row exchange between time steps.  With Phi lagged (or
// no G) the exchange follows the in-place AA pattern: a step from an even
// level touches only each node's own populations, so it needs nothing from the
// neighbours but the previous level's Phi_yyy row (for d_y Phi_yyy of G_i,
// eq_Gi); a step from an odd level reads the populations its neighbour row left
// in it and pushes populations into that row, so the boundary rows' y-moving
// slots are copied into the halo rows before it and back out of them after it.
// With Phi at the current level the two-buffer step computes Phi of every
// neighbour from its populations, so all nine populations of each boundary row
// go into the facing halo row before the step (the halo node's Phi is then the
// one the undivided lattice computes), and what the step pushed into the halo
// rows goes back to the rows that own it afterwards.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "lb_device.cuh"
#include "lb_handle.h"

struct trtrlb_slabs {
    trtrlb_params p;
    cudaStream_t stream = nullptr;
    std::vector<trtrlb_t> slab;     // bottom to top
    std::vector<int> row0;          // first global row owned by each slab
    std::vector<int> rows;          // rows owned by each slab
    std::vector<int> lo_halo;       // slab has a halo row below (local row 0)
    std::vector<int> hi_halo;       // slab has a halo row above
    char err[256] = "";
};

namespace {

int cuda_fail(trtrlb_slabs* s, cudaError_t e, const char* where) {
    std::snprintf(s->err, sizeof s->err, "%s: %s", where, cudaGetErrorString(e));
    return TRTRLB_ECUDA;
}

int lattice_fail(trtrlb_slabs* s, trtrlb_t h, int rc) {
    std::snprintf(s->err, sizeof s->err, "slab: %s", trtrlb_last_error(h));
    return rc;
}

size_t pop_bytes(int storage) {
    switch (storage) {
        case TRTRLB_F64: case TRTRLB_F64_DW: return 8;
        case TRTRLB_F32: return 4;
        default: return 2;
    }
}

size_t phi_bytes(int storage) {
    return (storage == TRTRLB_F64 || storage == TRTRLB_F64_DW) ? 8 : 4;
}

// Local row (in its slab) of the row just below / above slab k's owned rows.
int local_first(const trtrlb_slabs* s, int k) { return s->lo_halo[k]; }
int local_last(const trtrlb_slabs* s, int k) { return s->lo_halo[k] + s->rows[k] - 1; }

// Copies row `src_row` of planes `planes` of slab a's current populations into
// row `dst_row` of slab b.
template <int NP>
cudaError_t copy_pops(trtrlb_slabs* s, trtrlb_t a, int src_row, trtrlb_t b, int dst_row,
                      const int (&planes)[NP]) {
    const size_t es = pop_bytes(s->p.storage);
    const size_t row = (size_t)s->p.nx * es;
    for (int q : planes) {
        const char* src = static_cast<const char*>(a->s.f) + ((size_t)q * a->s.plane + (size_t)src_row * a->s.pitch) * es;
        char* dst = static_cast<char*>(b->s.f) + ((size_t)q * b->s.plane + (size_t)dst_row * b->s.pitch) * es;
        const cudaError_t e = cudaMemcpyAsync(dst, src, row, cudaMemcpyDefault, s->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Phi_yyy of the previous level (the Phi buffer the next step reads).
cudaError_t copy_phi_y(trtrlb_slabs* s, trtrlb_t a, int src_row, trtrlb_t b, int dst_row) {
    const size_t ps = phi_bytes(s->p.storage);
    const char* src = static_cast<const char*>(a->s.phi[a->s.cur]) + ((size_t)a->s.plane + (size_t)src_row * a->s.pitch) * ps;
    char* dst = static_cast<char*>(b->s.phi[b->s.cur]) + ((size_t)b->s.plane + (size_t)dst_row * b->s.pitch) * ps;
    return cudaMemcpyAsync(dst, src, (size_t)s->p.nx * ps, cudaMemcpyDefault, s->stream);
}

constexpr int kUp[3] = {2, 5, 6};     // e_y = +1
constexpr int kDown[3] = {4, 7, 8};   // e_y = -1
constexpr int kAll[9] = {0, 1, 2, 3, 4, 5, 6, 7, 8};

// Copies the slots (i, x) of one halo row that the step's push wrote, i in
// {i0, i1, i2}: those whose writer, the node x - e_i of the facing boundary
// row, lies inside the lattice and collides.  (The other slots of the owner's
// row hold what the owner wrote itself, e.g. bounce-back at a wall.)
template <typename T>
__global__ void k_halo_out(const T* __restrict__ src, T* __restrict__ dst, long long src_plane,
                           long long dst_plane, long long src_row, long long dst_row,
                           const uint8_t* __restrict__ writer_class, int i0, int i1, int i2, int nx,
                           int px) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    const int i = blockIdx.y == 0 ? i0 : (blockIdx.y == 1 ? i1 : i2);
    int w = x - trt::ex(i);
    if (w < 0 || w >= nx) {
        if (!px) return;
        w = w < 0 ? w + nx : w - nx;
    }
    if (writer_class && !trt::collides(writer_class[w])) return;
    dst[i * dst_plane + dst_row + x] = src[i * src_plane + src_row + x];
}

template <typename T>
cudaError_t launch_out(trtrlb_slabs* s, trtrlb_t a, int a_row, trtrlb_t b, int b_row, trtrlb_t writer,
                       int w_row, const int (&planes)[3]) {
    const dim3 block(128), grid((s->p.nx + 127) / 128, 3);
    const uint8_t* wc = writer->s.mask ? writer->s.mask + (size_t)w_row * writer->s.pitch : nullptr;
    k_halo_out<T><<<grid, block, 0, s->stream>>>(
        static_cast<const T*>(a->s.f), static_cast<T*>(b->s.f), a->s.plane, b->s.plane,
        (long long)a_row * a->s.pitch, (long long)b_row * b->s.pitch, wc, planes[0], planes[1],
        planes[2], s->p.nx, s->p.periodic_x);
    return cudaGetLastError();
}

// The populations the push of `writer`'s row w_row left in row a_row of a go
// to row b_row of b.
cudaError_t copy_out(trtrlb_slabs* s, trtrlb_t a, int a_row, trtrlb_t b, int b_row, trtrlb_t writer,
                     int w_row, const int (&planes)[3]) {
    switch (pop_bytes(s->p.storage)) {
        case 8: return launch_out<unsigned long long>(s, a, a_row, b, b_row, writer, w_row, planes);
        case 4: return launch_out<unsigned int>(s, a, a_row, b, b_row, writer, w_row, planes);
        default: return launch_out<unsigned short>(s, a, a_row, b, b_row, writer, w_row, planes);
    }
}

// The exchange across every interface (slab k below, slab u above).
//   PHI: the previous level's Phi_yyy of each boundary row into the facing halo
//        row (read by d_y Phi_yyy of the next step, LAGGED);
//   IN:  at an odd level, each boundary row's y-moving populations into the
//        facing halo row: an odd-level state keeps f_i(x) with e_iy = -1 of a
//        top row in the e_y = +1 slots of the row above (and the converse), so
//        both the next step's pull and any read of the state need them;
//   OUT: after a step from an odd level, or after a two-buffer step (Phi at
//        the current level), what the push left in each halo row (the e_y = +1
//        slots above a top row, e_y = -1 below a bottom row) back into the row
//        that owns it, slot by slot where the push wrote;
//   ROWS: before a two-buffer step, all nine populations of each boundary row
//        into the facing halo row.
enum Part { PHI, IN, OUT, ROWS };

cudaError_t exchange(trtrlb_slabs* s, Part part) {
    const int n = (int)s->slab.size();
    for (int k = 0; k < n; ++k) {
        if (!s->hi_halo[k]) continue;
        const int u = (k + 1) % n;
        trtrlb_t A = s->slab[k], B = s->slab[u];
        const int a_top = local_last(s, k), a_halo = a_top + 1;
        const int b_bot = local_first(s, u), b_halo = b_bot - 1;
        cudaError_t e = cudaSuccess;
        if (part == PHI) {
            e = copy_phi_y(s, B, b_bot, A, a_halo);
            if (e == cudaSuccess) e = copy_phi_y(s, A, a_top, B, b_halo);
        } else if (part == IN) {
            e = copy_pops(s, B, b_bot, A, a_halo, kUp);
            if (e == cudaSuccess) e = copy_pops(s, A, a_top, B, b_halo, kDown);
        } else if (part == ROWS) {
            e = copy_pops(s, B, b_bot, A, a_halo, kAll);
            if (e == cudaSuccess) e = copy_pops(s, A, a_top, B, b_halo, kAll);
        } else {
            e = copy_out(s, A, a_halo, B, b_bot, A, a_top, kUp);
            if (e == cudaSuccess) e = copy_out(s, B, b_halo, A, a_top, B, b_bot, kDown);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool odd_level(const trtrlb_slabs* s) { return s->slab[0]->s.parity != 0; }

// Makes the halo rows hold what a read of the current state needs.
cudaError_t sync_for_read(trtrlb_slabs* s) {
    return odd_level(s) ? exchange(s, IN) : cudaSuccess;
}

}  // namespace

extern "C" {

int trtrlb_slabs_create(const trtrlb_params* pp, const uint8_t* mask, int32_t nslabs, void* stream,
                        trtrlb_slabs_t* out) {
    if (!pp || !out || nslabs < 1) return TRTRLB_EINVAL;
    const trtrlb_params p = *pp;
    if (p.ny < nslabs || p.nx < 1) return TRTRLB_EINVAL;
    if (mask) {
        for (long long k = 0; k < (long long)p.nx * p.ny; ++k)
            if (mask[k] == TRTRLB_OUTLET || mask[k] == TRTRLB_HALO || mask[k] == TRTRLB_HALO_PRESSURE)
                return TRTRLB_ENOTSUP;
    }
    trtrlb_slabs* s = new (std::nothrow) trtrlb_slabs();
    if (!s) return TRTRLB_ENOMEM;
    s->p = p;
    s->stream = static_cast<cudaStream_t>(stream);
    const bool py = p.periodic_y != 0;
    int y = 0;
    for (int k = 0; k < nslabs; ++k) {
        const int r = p.ny / nslabs + (k < p.ny % nslabs ? 1 : 0);
        s->row0.push_back(y);
        s->rows.push_back(r);
        s->lo_halo.push_back(nslabs > 1 && (k > 0 || py) ? 1 : 0);
        s->hi_halo.push_back(nslabs > 1 && (k < nslabs - 1 || py) ? 1 : 0);
        y += r;
    }
    for (int k = 0; k < nslabs; ++k) {
        trtrlb_params q = p;
        const int lo = s->lo_halo[k], hi = s->hi_halo[k];
        q.ny = s->rows[k] + lo + hi;
        if (nslabs > 1) q.periodic_y = 0;
        std::vector<uint8_t> m((size_t)p.nx * q.ny, TRTRLB_FLUID);
        auto global_class = [&](int gy, int x) -> uint8_t {
            gy = (gy + p.ny) % p.ny;
            return mask ? mask[(long long)gy * p.nx + x] : (uint8_t)TRTRLB_FLUID;
        };
        for (int r = 0; r < q.ny; ++r) {
            const int gy = s->row0[k] - lo + r;
            const bool halo = (lo && r == 0) || (hi && r == q.ny - 1);
            for (int x = 0; x < p.nx; ++x) {
                uint8_t c = global_class(gy, x);
                // a halo node stands for a node another slab updates (a pressure
                // outlet node keeps its Zou-He rebuild for Phi); walls and
                // moving walls keep their class (they do not update anyway)
                if (halo && c == TRTRLB_FLUID) c = TRTRLB_HALO;
                else if (halo && c == TRTRLB_PRESSURE) c = TRTRLB_HALO_PRESSURE;
                m[(size_t)r * p.nx + x] = c;
            }
        }
        trtrlb_t h = nullptr;
        const bool need_mask = nslabs > 1 || mask;
        const int rc = trtrlb_create(&q, need_mask ? m.data() : nullptr, stream, &h);
        if (rc != TRTRLB_OK) {
            trtrlb_slabs_destroy(s);
            return rc;
        }
        s->slab.push_back(h);
    }
    *out = s;
    return TRTRLB_OK;
}

int trtrlb_slabs_destroy(trtrlb_slabs_t s) {
    if (!s) return TRTRLB_OK;
    for (trtrlb_t h : s->slab) trtrlb_destroy(h);
    delete s;
    return TRTRLB_OK;
}

const char* trtrlb_slabs_last_error(trtrlb_slabs_t s) { return s ? s->err : ""; }

int32_t trtrlb_slabs_count(trtrlb_slabs_t s) { return s ? (int32_t)s->slab.size() : -1; }

int trtrlb_slabs_slab(trtrlb_slabs_t s, int32_t k, trtrlb_t* h, int32_t* row0, int32_t* rows,
                      int32_t* halo_below) {
    if (!s || k < 0 || k >= (int32_t)s->slab.size()) return TRTRLB_EINVAL;
    if (h) *h = s->slab[k];
    if (row0) *row0 = s->row0[k];
    if (rows) *rows = s->rows[k];
    if (halo_below) *halo_below = s->lo_halo[k];
    return TRTRLB_OK;
}

int trtrlb_slabs_init(trtrlb_slabs_t s, const double* rho, const double* ux, const double* uy) {
    if (!s || !ux || !uy) return TRTRLB_EINVAL;
    s->err[0] = 0;
    const int nx = s->p.nx;
    for (size_t k = 0; k < s->slab.size(); ++k) {
        trtrlb_t h = s->slab[k];
        const int lo = s->lo_halo[k], ny = h->p.ny;
        const size_t n = (size_t)nx * ny;
        // local fields: the owned rows, zeros in the halo rows (not used: halo
        // nodes do not collide)
        std::vector<double> buf(3 * n, 0.0);
        const double* src[3] = {rho, ux, uy};
        for (int q = 0; q < 3; ++q) {
            if (!src[q]) continue;
            const cudaError_t e = cudaMemcpy(buf.data() + q * n + (size_t)lo * nx,
                                             src[q] + (size_t)s->row0[k] * nx,
                                             (size_t)s->rows[k] * nx * sizeof(double), cudaMemcpyDefault);
            if (e != cudaSuccess) return cuda_fail(s, e, "slab fields");
        }
        if (rho)
            for (size_t i = 0; i < n; ++i)
                if ((int)(i / nx) < lo || (int)(i / nx) >= lo + s->rows[k]) buf[i] = s->p.rho0;
        const int rc = trtrlb_init(h, rho ? buf.data() : nullptr, buf.data() + n, buf.data() + 2 * n);
        if (rc != TRTRLB_OK) return lattice_fail(s, h, rc);
    }
    return TRTRLB_OK;
}

int trtrlb_slabs_step(trtrlb_slabs_t s, int64_t nsteps) {
    if (!s || nsteps < 0) return TRTRLB_EINVAL;
    s->err[0] = 0;
    if (s->p.g_mode == TRTRLB_G_CURRENT) {
        for (int64_t t = 0; t < nsteps; ++t) {
            cudaError_t e = exchange(s, ROWS);
            if (e != cudaSuccess) return cuda_fail(s, e, "halo exchange");
            for (trtrlb_t h : s->slab) {
                const int rc = trtrlb_step(h, 1);
                if (rc != TRTRLB_OK) return lattice_fail(s, h, rc);
            }
            e = exchange(s, OUT);
            if (e != cudaSuccess) return cuda_fail(s, e, "halo exchange");
        }
        return TRTRLB_OK;
    }
    for (int64_t t = 0; t < nsteps; ++t) {
        const bool odd = odd_level(s);
        cudaError_t e = s->p.g_mode == TRTRLB_G_LAGGED ? exchange(s, PHI) : cudaSuccess;
        if (e == cudaSuccess && odd) e = exchange(s, IN);
        if (e != cudaSuccess) return cuda_fail(s, e, "halo exchange");
        for (trtrlb_t h : s->slab) {
            const int rc = trtrlb_step(h, 1);
            if (rc != TRTRLB_OK) return lattice_fail(s, h, rc);
        }
        if (odd) e = exchange(s, OUT);
        if (e != cudaSuccess) return cuda_fail(s, e, "halo exchange");
    }
    return TRTRLB_OK;
}

int trtrlb_slabs_get_f(trtrlb_slabs_t s, double* f) {
    if (!s || !f) return TRTRLB_EINVAL;
    s->err[0] = 0;
    if (const cudaError_t se = sync_for_read(s); se != cudaSuccess) return cuda_fail(s, se, "halo exchange");
    const size_t nx = (size_t)s->p.nx, n = nx * s->p.ny;
    for (size_t k = 0; k < s->slab.size(); ++k) {
        trtrlb_t h = s->slab[k];
        const size_t nl = nx * h->p.ny;
        std::vector<double> buf(9 * nl);
        const int rc = trtrlb_get_f(h, buf.data(), nullptr);
        if (rc != TRTRLB_OK) return lattice_fail(s, h, rc);
        for (int i = 0; i < 9; ++i) {
            const cudaError_t e = cudaMemcpy(f + i * n + (size_t)s->row0[k] * nx,
                                             buf.data() + i * nl + (size_t)s->lo_halo[k] * nx,
                                             (size_t)s->rows[k] * nx * sizeof(double), cudaMemcpyDefault);
            if (e != cudaSuccess) return cuda_fail(s, e, "get_f");
        }
    }
    return TRTRLB_OK;
}

int trtrlb_slabs_moments(trtrlb_slabs_t s, double* rho, double* ux, double* uy) {
    if (!s) return TRTRLB_EINVAL;
    s->err[0] = 0;
    if (const cudaError_t se = sync_for_read(s); se != cudaSuccess) return cuda_fail(s, se, "halo exchange");
    const size_t nx = (size_t)s->p.nx;
    double* dst[3] = {rho, ux, uy};
    for (size_t k = 0; k < s->slab.size(); ++k) {
        trtrlb_t h = s->slab[k];
        const size_t nl = nx * h->p.ny;
        std::vector<double> buf(3 * nl);
        const int rc = trtrlb_moments(h, buf.data(), buf.data() + nl, buf.data() + 2 * nl);
        if (rc != TRTRLB_OK) return lattice_fail(s, h, rc);
        for (int q = 0; q < 3; ++q) {
            if (!dst[q]) continue;
            const cudaError_t e = cudaMemcpy(dst[q] + (size_t)s->row0[k] * nx,
                                             buf.data() + q * nl + (size_t)s->lo_halo[k] * nx,
                                             (size_t)s->rows[k] * nx * sizeof(double), cudaMemcpyDefault);
            if (e != cudaSuccess) return cuda_fail(s, e, "moments");
        }
    }
    return TRTRLB_OK;
}

int trtrlb_slabs_diagnostics(trtrlb_slabs_t s, double* out) {
    if (!s || !out) return TRTRLB_EINVAL;
    s->err[0] = 0;
    if (const cudaError_t se = sync_for_read(s); se != cudaSuccess) return cuda_fail(s, se, "halo exchange");
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (trtrlb_t h : s->slab) {
        double d[8];
        const int rc = trtrlb_diagnostics(h, d);
        if (rc != TRTRLB_OK) return lattice_fail(s, h, rc);
        for (int q = 0; q < 8; ++q) acc[q] = q == 4 ? (d[q] > acc[q] ? d[q] : acc[q]) : acc[q] + d[q];
    }
    const cudaError_t e = cudaMemcpy(out, acc, sizeof acc, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(s, e, "diagnostics");
    return TRTRLB_OK;
}

}  // extern "C"
