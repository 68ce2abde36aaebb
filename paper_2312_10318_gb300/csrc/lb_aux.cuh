// Auxiliary kernels of the D2Q9 TRT-RLB library: initial state, static Phi
// values, moments, population import/export and FP64 diagnostics.  All of them
// read and write the AA storage through pop_loc (lb_device.cuh).
#pragma once
#include "lb_device.cuh"
#include "lb_ops.cuh"

#include <type_traits>
#include <utility>

namespace trt {

// Arithmetic of the import/export kernels (k_init, k_moments): FP64 for FP64
// storage, double-word FP32 (about 48 significant bits, lb_dw.cuh) for every
// other format, so that these kernels run on the FP32 pipes, which GB300 has
// many times more of than FP64 ones.
__device__ __forceinline__ void aux_round(df64 v, float& o) { o = __fadd_rn(v.hi, v.lo); }
__device__ __forceinline__ void aux_round(df64 v, df64& o) { o = v; }
__device__ __forceinline__ df64 aux_widen(float v) { return df64(v, 0.f); }
__device__ __forceinline__ df64 aux_widen(const df64& v) { return v; }
// c x for c in {-1, 0, 1} known at compile time once the loops are unrolled
template <typename A>
__device__ __forceinline__ A aux_sel(int c, const A& x) {
    return c > 0 ? x : (c < 0 ? -x : A(0));
}

// A double-word constant, split at compile time (no FP64 instruction runs).
__host__ __device__ constexpr df64 dw_const(double x) {
    return df64((float)x, (float)(x - (double)(float)x));
}

// Direction I of the initial state in double-word arithmetic (k_init), its
// lattice constants fixed at compile time.
template <int I, typename S>
__device__ __forceinline__ void init_dir(S* F, long long plane, long long own, const df64& r, const df64& u,
                                         const df64& v, const df64& uu, const df64& vv, const df64& uv,
                                         const df64& uuv, const df64& uvv, const df64& Fx, const df64& Fy,
                                         const df64& r0) {
    using A = df64;
    using C = typename Fmt<S>::C;
    constexpr int cx = ex(I), cy = ey(I);
    constexpr A KX = dw_const(cx * cx - 1.0 / 3.0), KY = dw_const(cy * cy - 1.0 / 3.0);
    constexpr A W = dw_const(wgt(I)), W15 = dw_const(1.5 * wgt(I));
    constexpr A ONE = dw_const(1.0), THREE = dw_const(3.0), K45 = dw_const(4.5), K135 = dw_const(13.5);
    const A eu = aux_sel(cx, u) + aux_sel(cy, v);
    A huu = KX * uu + KY * vv;
    if constexpr (cx * cy != 0) huu = huu + aux_sel(cx * cy, uv + uv);
    const A h3 = aux_sel(cy, KX * uuv) + aux_sel(cx, KY * uvv);
    const A feq = W * r * (ONE + THREE * eu + K45 * huu + K135 * h3);
    const A eF = aux_sel(cx, Fx) + aux_sel(cy, Fy);
    C out;
    aux_round(feq - W15 * eF - W * r0, out);
    F[(long long)I * plane + own] = Fmt<S>::st(out);
}

template <typename S, int... I>
__device__ __forceinline__ void init_dirs(std::integer_sequence<int, I...>, S* F, long long plane, long long own,
                                          const df64& r, const df64& u, const df64& v, const df64& uu,
                                          const df64& vv, const df64& uv, const df64& uuv, const df64& uvv,
                                          const df64& Fx, const df64& Fy, const df64& r0) {
    (init_dir<I, S>(F, plane, own, r, u, v, uu, vv, uv, uuv, uvv, Fx, Fy, r0), ...);
}

// Direction I of the initial state for FP32 and 16-bit storage (k_init):
// d_i = w_i [drho + 3 e_i.(rho u) + T], T in FP32.
template <int I, typename S>
__device__ __forceinline__ void init_dir_mixed(S* F, long long plane, long long own, const df64& dr,
                                               const df64& ru, const df64& rv, float rf, float uf, float vf,
                                               float gx, float gy) {
    using C = typename Fmt<S>::C;
    constexpr int cx = ex(I), cy = ey(I);
    constexpr float kx = (float)(cx * cx) - 1.0f / 3.0f, ky = (float)(cy * cy) - 1.0f / 3.0f;
    constexpr df64 W = dw_const(wgt(I));
    const df64 eru = aux_sel(cx, ru) + aux_sel(cy, rv);            // e_i.(rho u)
    df64 s3;                                                        // 3 e_i.(rho u), exact scaling by 3
    two_prod(eru.hi, 3.0f, s3.hi, s3.lo);
    s3.lo = fmaf(eru.lo, 3.0f, s3.lo);
    fast_two_sum(s3.hi, s3.lo, s3.hi, s3.lo);
    const float huu = kx * uf * uf + ky * vf * vf + (float)(2 * cx * cy) * uf * vf;
    const float h3 = kx * (float)cy * uf * uf * vf + ky * (float)cx * uf * vf * vf;
    const float t = rf * (4.5f * huu + 13.5f * h3 - 1.5f * ((float)cx * gx + (float)cy * gy));
    df64 sum = dr + s3;
    float sh, sl;
    two_sum(sum.hi, t, sh, sl);
    fast_two_sum(sh, __fadd_rn(sl, sum.lo), sum.hi, sum.lo);
    C out;
    aux_round(W * sum, out);
    F[(long long)I * plane + own] = Fmt<S>::st(out);
}

template <typename S, int... I>
__device__ __forceinline__ void init_dirs_mixed(std::integer_sequence<int, I...>, S* F, long long plane,
                                                long long own, const df64& dr, const df64& ru, const df64& rv,
                                                float rf, float uf, float vf, float gx, float gy) {
    (init_dir_mixed<I, S>(F, plane, own, dr, ru, rv, rf, uf, vf, gx, gy), ...);
}

// Phi of non-fluid nodes (reading of the paper's silence on walls): 0 at
// solid nodes, rho_w u_w^3 at moving-wall (inlet) nodes.  Both buffers.
template <typename C>
__global__ void k_phi_static(const uint8_t* __restrict__ mask, int nx, int ny, int pitch,
                             long long plane, C* phi0, C* phi1, C inx, C iny) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long k = (long long)y * pitch + x;
    const uint8_t c = mask ? mask[k] : FLUID;
    if (collides(c) || c == OUTLET) return;
    const C vx = c == INLET ? inx : C(0), vy = c == INLET ? iny : C(0);
    phi0[k] = vx; phi0[plane + k] = vy;
    phi1[k] = vx; phi1[plane + k] = vy;
}

// Phi(s) := Phi(s - (1,0)) for every outlet ghost s, in one buffer.
template <typename C>
__global__ void k_ghost_phi(const int* __restrict__ ghosts, int nghost, int nx, int pitch,
                            long long plane, C* phi) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nghost) return;
    const int s = ghosts[g];
    const int sx = s % pitch, sy = s / pitch;
    int zx = sx - 1;
    if (zx < 0) zx += nx;
    const long long z = (long long)sy * pitch + zx;
    phi[s] = phi[z];
    phi[plane + s] = phi[plane + z];
}

// Initial state at an even level (reading of the paper's silence on
// initialisation): f_i = f_i^eq(rho, u) - (1/2) w_i e_i.F / c_s^2 with the
// third-order equilibrium of eq4 and F = rho g, so that sum f = rho and
// sum e f = rho u - F/2 (eq11).  Arithmetic in FP64 (FP64 storage) or
// double-word FP32 (the other formats), rounded once to S.
// Also Phi = (rho u_x^3, rho u_y^3) into both buffers (Phi^{-1} := Phi^0).
template <typename S>
__global__ void k_init(Args<typename Fmt<S>::C> a, const double* __restrict__ rho,
                       const double* __restrict__ ux, const double* __restrict__ uy, double rho0,
                       double gx, double gy, typename Fmt<S>::C* phi_b) {
    using C = typename Fmt<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    S* F = static_cast<S*>(a.f);
    const long long own = (long long)y * a.pitch + x;
    const long long k = (long long)y * a.nx + x;
    const bool fluid = !a.mask || collides(a.mask[own]);
    if (!fluid) {
#pragma unroll
        for (int i = 0; i < 9; ++i) F[(long long)i * a.plane + own] = Fmt<S>::st(C(0));
        return;
    }
    if constexpr (std::is_same<S, double>::value) {
        const double r = rho ? rho[k] : rho0;
        const double u = ux[k], v = uy[k];
        const double t = 1.0 / 3.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double cx = ex(i), cy = ey(i), w = wgt(i);
            const double eu = cx * u + cy * v;
            const double huu = (cx * cx - t) * u * u + 2.0 * cx * cy * u * v + (cy * cy - t) * v * v;
            const double h3 = (cx * cx - t) * cy * u * u * v + (cy * cy - t) * cx * u * v * v;
            const double feq = w * r * (1.0 + 3.0 * eu + 4.5 * huu + 13.5 * h3);
            const double eF = r * (cx * gx + cy * gy);
            F[(long long)i * a.plane + own] = Fmt<S>::st((C)(feq - 1.5 * w * eF - w * rho0));
        }
        const C px = (C)(r * u * u * u), py = (C)(r * v * v * v);
        a.phi_out[own] = px; a.phi_out[a.plane + own] = py;
        phi_b[own] = px; phi_b[a.plane + own] = py;
    } else if constexpr (!std::is_same<S, f64dw>::value) {
        // FP32 and the 16-bit formats, whose stores round to 2^-24 or coarser:
        // d_i / w_i = drho + 3 e_i.(rho u) + rho (4.5 H:uu + 13.5 H3:uuu
        // - 1.5 e_i.g), the first two terms (up to ~0.3) in double-word
        // arithmetic, the rest (|.| <~ 0.1 rho) in FP32, whose error there,
        // 2^-24 of it, stays below one rounding of the stored value; the inputs
        // split without FP64 instructions
        using A = df64;
        const A r = df64_split(rho ? rho[k] : rho0);
        const A u = df64_split(ux[k]), v = df64_split(uy[k]);
        const A dr = rho ? r - df64_split(rho0) : A(0.f, 0.f);
        const A ru = r * u, rv = r * v;
        const float rf = r.hi, uf = u.hi, vf = v.hi;
        const float fgx = a.gx, fgy = a.gy;   // the FP32 arguments: no conversion per node
        init_dirs_mixed<S>(std::make_integer_sequence<int, 9>{}, F, a.plane, own, dr, ru, rv, rf, uf, vf, fgx, fgy);
        C px, py;
        aux_round(r * (u * u) * u, px);
        aux_round(r * (v * v) * v, py);
        a.phi_out[own] = px; a.phi_out[a.plane + own] = py;
        phi_b[own] = px; phi_b[a.plane + own] = py;
    } else {
        // the same equilibrium, with the velocity products shared by the directions
        using A = df64;
        auto in = [](double x) { return A(x); };
        const A r = in(rho ? rho[k] : rho0);
        const A u = in(ux[k]), v = in(uy[k]);
        const A uu = u * u, vv = v * v, uv = u * v, uuv = uu * v, uvv = u * vv;
        const A Fx = r * in(gx), Fy = r * in(gy), r0 = in(rho0);
        init_dirs<S>(std::make_integer_sequence<int, 9>{}, F, a.plane, own, r, u, v, uu, vv, uv, uuv, uvv, Fx,
                     Fy, r0);
        C px, py;
        aux_round(r * uu * u, px);
        aux_round(r * vv * v, py);
        a.phi_out[own] = px; a.phi_out[a.plane + own] = py;
        phi_b[own] = px; phi_b[a.plane + own] = py;
    }
}

// FP64 moments (eq11) of a state of parity ODD into dense [ny][nx] arrays;
// any output may be null; non-fluid nodes give 0.  Computed in FP64 for FP64
// storage and in double-word FP32 (about 48 bits) for the other formats.
template <typename S, bool ODD>
__global__ void k_moments(Args<typename Fmt<S>::C> a, double* rho, double* ux, double* uy) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const S* F = static_cast<const S*>(a.f);
    const long long own = (long long)y * a.pitch + x;
    const long long k = (long long)y * a.nx + x;
    const int c = a.mask ? a.mask[own] : FLUID;
    if (!collides(c)) {
        if (rho) rho[k] = 0.0;
        if (ux) ux[k] = 0.0;
        if (uy) uy[k] = 0.0;
        return;
    }
    int nb[9];
    int kind[9];
    links<true>(a, x, y, nb, kind);
    if constexpr (std::is_same<S, double>::value) {
        double d[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = Fmt<S>::ld(F[pop_loc<ODD>(a.plane, nb, kind, i)]);
        if (c == PRESSURE) zh_fill<double>(d, a.zh_dr);
        double r, u, v;
        moments_of<double>(d, a.gx, a.gy, a.rho0, r, u, v);
        if (rho) rho[k] = r;
        if (ux) ux[k] = u;
        if (uy) uy[k] = v;
    } else {
        df64 d[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = aux_widen(Fmt<S>::ld(F[pop_loc<ODD>(a.plane, nb, kind, i)]));
        if (c == PRESSURE) zh_fill<df64>(d, aux_widen(a.zh_dr));
        df64 r, u, v;
        moments_of<df64>(d, aux_widen(a.gx), aux_widen(a.gy), aux_widen(a.rho0), r, u, v);
        if (rho) rho[k] = dw_to_double(r);
        if (ux) ux[k] = dw_to_double(u);
        if (uy) uy[k] = dw_to_double(v);
    }
}

// Export f_i(x, t) as FP64 [9][ny][nx] (non-fluid: 0) and Phi_in as [2][ny][nx].
template <typename S, bool ODD>
__global__ void k_get_f(Args<typename Fmt<S>::C> a, double* f, double* phi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const S* F = static_cast<const S*>(a.f);
    const long long own = (long long)y * a.pitch + x;
    const long long k = (long long)y * a.nx + x, n = (long long)a.nx * a.ny;
    if (phi) {
        phi[k] = (double)a.phi_in[own];
        phi[n + k] = (double)a.phi_in[a.plane + own];
    }
    if (!f) return;
    const int c = a.mask ? a.mask[own] : FLUID;
    if (!collides(c)) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i * n + k] = 0.0;
        return;
    }
    int nb[9];
    int kind[9];
    links<true>(a, x, y, nb, kind);
    double d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = (double)Fmt<S>::ld(F[pop_loc<ODD>(a.plane, nb, kind, i)]);
    if (c == PRESSURE) zh_fill<double>(d, (double)a.zh_dr);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i * n + k] = d[i] + wgt(i) * (double)a.rho0;
}

// Import f_i(x, t) (FP64 [9][ny][nx]) as an even-level state; fluid nodes only.
// phi (optional, [2][ny][nx]) is copied into Phi_in for every node.
template <typename S>
__global__ void k_set_f(Args<typename Fmt<S>::C> a, const double* f, const double* phi) {
    using C = typename Fmt<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    S* F = static_cast<S*>(a.f);
    C* P = const_cast<C*>(a.phi_in);
    const long long own = (long long)y * a.pitch + x;
    const long long k = (long long)y * a.nx + x, n = (long long)a.nx * a.ny;
    if (phi) {
        P[own] = (C)phi[k];
        P[a.plane + own] = (C)phi[n + k];
    }
    if (a.mask && !collides(a.mask[own])) return;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        F[(long long)i * a.plane + own] = Fmt<S>::st((C)(f[i * n + k] - wgt(i) * (double)a.rho0));
}

// Phi_in of the fluid nodes from the moments of an even-level state.
template <typename S>
__global__ void k_phi_of_state(Args<typename Fmt<S>::C> a) {
    using C = typename Fmt<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    const S* F = static_cast<const S*>(a.f);
    C* P = const_cast<C*>(a.phi_in);
    const long long own = (long long)y * a.pitch + x;
    const int c = a.mask ? a.mask[own] : FLUID;
    if (!collides(c)) return;
    C d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = Fmt<S>::ld(F[(long long)i * a.plane + own]);
    if (c == PRESSURE) zh_fill<C>(d, a.zh_dr);
    C r, u, v;
    moments_of<C>(d, a.gx, a.gy, a.rho0, r, u, v);
    P[own] = r * u * u * u;
    P[a.plane + own] = r * v * v * v;
}

// ---- FP64 diagnostics: deterministic two-level reduction --------------------
constexpr int NDIAG = 8;

struct Diag {
    double v[NDIAG];  // mass, momentum x, y, kinetic energy, max|u|, non-finite, drag x, y
};

__device__ __forceinline__ void diag_merge(Diag& a, const Diag& b) {
#pragma unroll
    for (int q = 0; q < NDIAG; ++q) a.v[q] = (q == 4) ? fmax(a.v[q], b.v[q]) : a.v[q] + b.v[q];
}

// Block tree reduction in a fixed order; thread 0 returns the block total.
__device__ __forceinline__ Diag diag_block_reduce(Diag d) {
    __shared__ double sh[NDIAG][DIAG_THREADS];
#pragma unroll
    for (int q = 0; q < NDIAG; ++q) sh[q][threadIdx.x] = d.v[q];
    __syncthreads();
    for (int s = DIAG_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
#pragma unroll
            for (int q = 0; q < NDIAG; ++q) {
                const double o = sh[q][threadIdx.x + s];
                sh[q][threadIdx.x] = (q == 4) ? fmax(sh[q][threadIdx.x], o) : sh[q][threadIdx.x] + o;
            }
        }
        __syncthreads();
    }
    Diag r;
#pragma unroll
    for (int q = 0; q < NDIAG; ++q) r.v[q] = sh[q][0];
    return r;
}

// Level 1: each block covers a fixed contiguous range of nodes (grid-stride
// order is fixed by the launch shape) and writes its partial to part[block].
template <typename S, bool ODD>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag_partial(Args<typename Fmt<S>::C> a,
                                                               double* __restrict__ part) {
    const S* F = static_cast<const S*>(a.f);
    const long long n = (long long)a.nx * a.ny;
    Diag acc;
#pragma unroll
    for (int q = 0; q < NDIAG; ++q) acc.v[q] = 0.0;
    for (long long k = (long long)blockIdx.x * DIAG_THREADS + threadIdx.x; k < n;
         k += (long long)gridDim.x * DIAG_THREADS) {
        const int x = (int)(k % a.nx), y = (int)(k / a.nx);
        const long long own = (long long)y * a.pitch + x;
        const int c = a.mask ? a.mask[own] : FLUID;
        if (!collides(c)) continue;
        int nb[9];
        int kind[9];
        links<true>(a, x, y, nb, kind);
        double d[9];
        bool finite = true;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            d[i] = (double)Fmt<S>::ld(F[pop_loc<ODD>(a.plane, nb, kind, i)]);
            finite = finite && isfinite(d[i]);
        }
        if (c == PRESSURE) zh_fill<double>(d, (double)a.zh_dr);
        if (!finite) {
            acc.v[5] += 1.0;
            continue;
        }
        double r, u, v;
        moments_of<double>(d, (double)a.gx, (double)a.gy, (double)a.rho0, r, u, v);
        acc.v[0] += r;
        acc.v[1] += r * u;
        acc.v[2] += r * v;
        acc.v[3] += 0.5 * r * (u * u + v * v);
        acc.v[4] = fmax(acc.v[4], sqrt(u * u + v * v));
        // momentum exchange with stationary walls: links into solid nodes or
        // across non-periodic edges carry 2 e_i f_ibar(x) (Sec. III D); the
        // links leaving a pressure outlet across the edge are open
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const bool wall = kind[i] == K_WALL && !(c == PRESSURE && ex(i) > 0);
            if (wall) {
                const double fr = d[opp(i)] + wgt(opp(i)) * (double)a.rho0;
                acc.v[6] += 2.0 * ex(i) * fr;
                acc.v[7] += 2.0 * ey(i) * fr;
            }
        }
    }
    const Diag tot = diag_block_reduce(acc);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NDIAG; ++q) part[(long long)blockIdx.x * NDIAG + q] = tot.v[q];
    }
}

// Level 2: one block folds the partials in a fixed order.
static __global__ void __launch_bounds__(DIAG_THREADS) k_diag_final(const double* __restrict__ part,
                                                             int nblocks, double* out) {
    Diag acc;
#pragma unroll
    for (int q = 0; q < NDIAG; ++q) acc.v[q] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += DIAG_THREADS) {
        Diag p;
#pragma unroll
        for (int q = 0; q < NDIAG; ++q) p.v[q] = part[(long long)b * NDIAG + q];
        diag_merge(acc, p);
    }
    const Diag tot = diag_block_reduce(acc);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NDIAG; ++q) out[q] = tot.v[q];
    }
}

}  // namespace trt
