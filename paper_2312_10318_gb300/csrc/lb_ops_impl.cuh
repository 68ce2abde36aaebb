// Definitions of Ops<S> (lb_ops.cuh); included once per storage format.
#pragma once
#include <type_traits>

#include "lb_ab.cuh"
#include "lb_ab_col.cuh"
#include "lb_ab_tma.cuh"
#include "lb_aux.cuh"
#include "lb_batch.cuh"
#include "lb_ops.cuh"

namespace trt {

template <typename C>
static Args<C> make_args(const State& s, bool swap_phi = false) {
    Args<C> a;
    a.f = s.f;
    const int in = swap_phi ? 1 - s.cur : s.cur;
    a.phi_in = static_cast<const C*>(s.phi[in]);
    a.phi_out = static_cast<C*>(s.phi[1 - in]);
    a.mask = s.mask;
    a.seg = s.seg;
    a.segs = s.segs;
    a.nx = s.nx; a.ny = s.ny; a.pitch = s.pitch; a.plane = s.plane;
    a.px = s.px; a.py = s.py;
    const double k1 = 1.0 - 1.0 / s.tau1, k2 = 1.0 - 1.0 / s.tau2;
    a.k1 = (C)k1;
    a.k1lo = (C)(k1 - (double)a.k1);   // 0 when C is double
    a.k2 = (C)k2;
    a.k2lo = (C)(k2 - (double)a.k2);
    a.kf = (C)(1.0 - 1.0 / (2.0 * s.tau1));
    a.gx = (C)s.gx; a.gy = (C)s.gy; a.rho0 = (C)s.rho0;
    for (int i = 0; i < 9; ++i) {
        // 2 w_i rho_w (e_i.u_w) / c_s^2, subtracted from f*_i when e_i points
        // into a moving wall (Ladd's correction)
        const double eu = ex(i) * s.wall_ux + ey(i) * s.wall_uy;
        a.corr[i] = (C)(6.0 * wgt(i) * s.wall_rho * eu);
    }
    a.phin_x = (C)(s.wall_rho * s.wall_ux * s.wall_ux * s.wall_ux);
    a.phin_y = (C)(s.wall_rho * s.wall_uy * s.wall_uy * s.wall_uy);
    a.zh_dr = (C)(s.rho0 - s.outlet_rho);
    return a;
}

static inline dim3 grid2d(const State& s, dim3 b) {
    return dim3((s.nx + b.x - 1) / b.x, (s.ny + b.y - 1) / b.y);
}

template <typename S, bool ODD>
static void launch_step(const State& s, const Args<typename Fmt<S>::C>& a, cudaStream_t st) {
    const int tw = s.tile_w > 0 ? s.tile_w : 128;
    const dim3 b(tw, 256 / tw);
    const dim3 g = grid2d(s, b);
    if (s.general) {
        if (s.g_mode == G_OFF) k_step<S, ODD, true, G_OFF><<<g, b, 0, st>>>(a);
        else k_step<S, ODD, true, G_LAGGED><<<g, b, 0, st>>>(a);
    } else {
        if (s.g_mode == G_OFF) k_step<S, ODD, false, G_OFF><<<g, b, 0, st>>>(a);
        else k_step<S, ODD, false, G_LAGGED><<<g, b, 0, st>>>(a);
    }
}

template <typename S, bool ODD>
static void launch_step_vec(const State& s, const Args<typename Fmt<S>::C>& a, cudaStream_t st) {
    constexpr int V = Pk<S>::V;
    const int spr = (s.nx + 32 * V - 1) / (32 * V);
    const long long nseg = (long long)spr * s.ny;
    const int blocks = (int)((nseg + 7) / 8);
    if (s.g_mode == G_OFF) k_step_vec<S, ODD, G_OFF><<<blocks, 256, 0, st>>>(a, spr);
    else k_step_vec<S, ODD, G_LAGGED><<<blocks, 256, 0, st>>>(a, spr);
}

template <typename S>
cudaError_t Ops<S>::step_ab(const State& s, int q, cudaStream_t st) {
    using C = typename Fmt<S>::C;
    State v = s;
    if (q & 1) {            // odd step of a sequence: the buffers have swapped
        v.f = s.f2;
        v.f2 = s.f;
    }
    if constexpr (std::is_same<S, float>::value) {
        if (tma_eligible(s)) {
            const State* one = &s;
            return step_ab_group(&one, 1, q, st);
        }
    }
    const Args<C> a = make_args<C>(v);
    if constexpr (!std::is_same<S, f64dw>::value) {
        if (s.col_h > 0 && !s.general) {
            const int gx = (s.nx + COL_W - 1) / COL_W, bands = (s.ny + s.col_h - 1) / s.col_h;
            const long long warps = (long long)gx * bands;
            const int blocks = (int)((warps + COL_WARPS - 1) / COL_WARPS);
            k_step_ab_col<S><<<blocks, COL_WARPS * 32, 0, st>>>(a, static_cast<S*>(v.f2), gx, bands, s.col_h);
            return cudaGetLastError();
        }
    }
    const dim3 g((s.nx + AB_TX - 1) / AB_TX, (s.ny + AB_TY - 1) / AB_TY);
    if (s.general) k_step_ab<S, true><<<g, AB_TX * AB_TY, 0, st>>>(a, static_cast<S*>(v.f2), 0);
    else k_step_ab<S, false><<<g, AB_TX * AB_TY, 0, st>>>(a, static_cast<S*>(v.f2), 0);
    return cudaGetLastError();
}

// Dynamic shared memory and carveout of a TMA kernel; occ becomes the smaller
// of its value and the kernel's resident CTAs per SM.
template <typename K>
static cudaError_t tma_setup(K kernel, int& occ) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TMA_SMEM_BYTES);
    // all of the unified L1/shared array as shared memory, so that the resident
    // CTAs the occupancy query counts are the ones that run (the grid is
    // persistent: one missing CTA per SM is a second wave)
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    int o = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, AB_TX * AB_TY, TMA_SMEM_BYTES);
    if (e == cudaSuccess) occ = occ == 0 || o < occ ? o : occ;
    return e;
}

template <typename S>
bool Ops<S>::tma_eligible(const State& s) {
    return std::is_same<S, float>::value && !s.general && s.g_mode == G_CURRENT && s.tma_grid > 0 &&
           s.kerr != nullptr;
}

// Member k of a TMA launch: lattice s at step q of a sequence (the buffers
// alternate with q, as in step_ab); returns its tile count.
template <int MAXL>
static int tma_member(TmaGroup<MAXL>& g, int k, const State& s, int q) {
    State v = s;
    if (q & 1) {
        v.f = s.f2;
        v.f2 = s.f;
    }
    const int buf = v.f == s.tma_buf[0] ? 0 : 1;
    g.map[k] = *static_cast<const CUtensorMap*>(s.tma_map[buf]);
    g.a[k] = make_args<float>(v);
    g.dst[k] = static_cast<float*>(v.f2);
    g.err[k] = s.kerr;
    g.tiles_x[k] = (s.nx + AB_TX - 1) / AB_TX;
    return g.tiles_x[k] * ((s.ny + TMA_TH - 1) / TMA_TH);
}

template <int MAXL>
static cudaError_t launch_tma(const State* const* m, int n, int q, cudaStream_t st) {
    TmaGroup<MAXL> g;
    g.n = n;
    g.tile_begin[0] = 0;
    int grid = 0;
    long long wait = 0;
    for (int k = 0; k < n; ++k) {
        g.tile_begin[k + 1] = g.tile_begin[k] + tma_member(g, k, *m[k], q);
        grid = k == 0 || m[k]->tma_grid < grid ? m[k]->tma_grid : grid;
        wait = k == 0 || m[k]->wait_limit < wait ? m[k]->wait_limit : wait;
    }
    const int ntiles = g.tile_begin[n];
    if (ntiles == 0) return cudaSuccess;
    k_step_ab_tma<MAXL><<<ntiles < grid ? ntiles : grid, AB_TX * AB_TY, TMA_SMEM_BYTES, st>>>(g, ntiles, wait);
    return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::step_ab_group(const State* const* members, int n, int q, cudaStream_t st) {
    if constexpr (std::is_same<S, float>::value) {
        for (int k = 0; k < n; ++k)
            if (!tma_eligible(*members[k])) return cudaErrorInvalidValue;
        if (n == 1) return launch_tma<1>(members, 1, q, st);
        for (int k0 = 0; k0 < n; k0 += TMA_GROUP_MAX) {
            const int c = n - k0 < TMA_GROUP_MAX ? n - k0 : TMA_GROUP_MAX;
            const cudaError_t e = launch_tma<TMA_GROUP_MAX>(members + k0, c, q, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    } else {
        (void)members; (void)n; (void)q; (void)st;
        return cudaErrorInvalidValue;
    }
}

template <typename S>
int Ops<S>::tma_grid() {
    if constexpr (std::is_same<S, float>::value) {
        int dev = 0, sms = 0, occ = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            tma_setup(k_step_ab_tma<1>, occ) != cudaSuccess ||
            tma_setup(k_step_ab_tma<TMA_GROUP_MAX>, occ) != cudaSuccess)
            return 0;
        return occ * sms;
    } else {
        return 0;
    }
}

template <typename S>
cudaError_t Ops<S>::step(State& s, cudaStream_t st) {
    using C = typename Fmt<S>::C;
    if (s.g_mode == G_CURRENT) {
        const cudaError_t e = step_ab(s, 0, st);
        void* t = s.f;
        s.f = s.f2;
        s.f2 = t;
        return e;
    }
    const Args<C> a = make_args<C>(s);
    if (s.vec) {
        if (s.parity == 0) launch_step_vec<S, false>(s, a, st);
        else launch_step_vec<S, true>(s, a, st);
    } else if (s.parity == 0) {
        launch_step<S, false>(s, a, st);
    } else {
        launch_step<S, true>(s, a, st);
    }
    if (s.nghost > 0) {
        const int t = 128, g = (s.nghost + t - 1) / t;
        if (s.parity == 0) k_ghosts<S, true><<<g, t, 0, st>>>(a, s.ghosts, s.nghost);
        else k_ghosts<S, false><<<g, t, 0, st>>>(a, s.ghosts, s.nghost);
    }
    s.parity ^= 1;
    if (s.g_mode == G_LAGGED) s.cur ^= 1;
    return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::phi_static(State& s, cudaStream_t st) {
    using C = typename Fmt<S>::C;
    cudaError_t e = cudaMemsetAsync(s.phi[0], 0, sizeof(C) * 2 * s.plane, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.phi[1], 0, sizeof(C) * 2 * s.plane, st);
    if (e != cudaSuccess) return e;
    if (!s.mask) return cudaSuccess;
    const dim3 b(32, 8);
    const C inx = (C)(s.wall_rho * s.wall_ux * s.wall_ux * s.wall_ux);
    const C iny = (C)(s.wall_rho * s.wall_uy * s.wall_uy * s.wall_uy);
    k_phi_static<C><<<grid2d(s, b), b, 0, st>>>(s.mask, s.nx, s.ny, s.pitch, s.plane,
                                                static_cast<C*>(s.phi[0]),
                                                static_cast<C*>(s.phi[1]), inx, iny);
    return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::init(State& s, const double* rho, const double* ux, const double* uy,
                         cudaStream_t st) {
    using C = typename Fmt<S>::C;
    s.parity = 0;
    s.cur = 0;
    const Args<C> a = make_args<C>(s, /*swap_phi=*/true);  // phi_out = phi[0] (the "in" level)
    const dim3 b(32, 8);
    k_init<S><<<grid2d(s, b), b, 0, st>>>(a, rho, ux, uy, s.rho0, s.gx, s.gy,
                                          static_cast<C*>(s.phi[1]));
    if (s.nghost > 0) {
        const int t = 128, g = (s.nghost + t - 1) / t;
        for (int q = 0; q < 2; ++q)
            k_ghost_phi<C><<<g, t, 0, st>>>(s.ghosts, s.nghost, s.nx, s.pitch, s.plane,
                                            static_cast<C*>(s.phi[q]));
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::moments(const State& s, double* rho, double* ux, double* uy,
                            cudaStream_t st) {
    using C = typename Fmt<S>::C;
    const Args<C> a = make_args<C>(s);
    const dim3 b(32, 8);
    if (s.parity) k_moments<S, true><<<grid2d(s, b), b, 0, st>>>(a, rho, ux, uy);
    else k_moments<S, false><<<grid2d(s, b), b, 0, st>>>(a, rho, ux, uy);
    return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::get_f(const State& s, double* f, double* phi, cudaStream_t st) {
    using C = typename Fmt<S>::C;
    const Args<C> a = make_args<C>(s);
    const dim3 b(32, 8);
    if (s.parity) k_get_f<S, true><<<grid2d(s, b), b, 0, st>>>(a, f, phi);
    else k_get_f<S, false><<<grid2d(s, b), b, 0, st>>>(a, f, phi);
    return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::set_f(State& s, const double* f, const double* phi, cudaStream_t st) {
    using C = typename Fmt<S>::C;
    s.parity = 0;
    const Args<C> a = make_args<C>(s);
    const dim3 b(32, 8);
    k_set_f<S><<<grid2d(s, b), b, 0, st>>>(a, f, phi);
    if (!phi) {
        k_phi_of_state<S><<<grid2d(s, b), b, 0, st>>>(a);
        if (s.nghost > 0) {
            const int t = 128, g = (s.nghost + t - 1) / t;
            k_ghost_phi<C><<<g, t, 0, st>>>(s.ghosts, s.nghost, s.nx, s.pitch, s.plane,
                                            static_cast<C*>(s.phi[s.cur]));
        }
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::diagnostics(const State& s, double* part, double* out, cudaStream_t st) {
    using C = typename Fmt<S>::C;
    const Args<C> a = make_args<C>(s);
    const int nb = diag_blocks(s);
    if (s.parity) k_diag_partial<S, true><<<nb, DIAG_THREADS, 0, st>>>(a, part);
    else k_diag_partial<S, false><<<nb, DIAG_THREADS, 0, st>>>(a, part);
    k_diag_final<<<1, DIAG_THREADS, 0, st>>>(part, nb, out);
    return cudaGetLastError();
}

// FLAV: FLAV_GENERAL, FLAV_PERIODIC (scalar kernels) or FLAV_VECTOR.
template <typename S, bool ODD, int FLAV, int GMODE, int MAXL>
static cudaError_t launch_group(const State* const* m, const int* cur, const int* l2tw, int n,
                                cudaStream_t st) {
    using C = typename Fmt<S>::C;
    constexpr int V = Pk<S>::V;
    GroupParams<C, MAXL> p;
    p.n = n;
    int tiles = 0;
    for (int q = 0; q < n; ++q) {
        State v = *m[q];
        v.cur = cur[q];
        p.a[q] = make_args<C>(v);
        p.tile_begin[q] = tiles;
        if (FLAV == FLAV_VECTOR) {
            p.segs[q] = (v.nx + 32 * V - 1) / (32 * V);
            p.inv_d[q] = 1.0f / (float)p.segs[q];
            p.tiles_x[q] = 0;
            p.log2_tw[q] = 0;
            tiles += (int)(((long long)p.segs[q] * v.ny + 7) / 8);
        } else {
            const int tw = 1 << l2tw[q], th = BATCH_THREADS / tw;
            p.log2_tw[q] = l2tw[q];
            p.segs[q] = 0;
            p.tiles_x[q] = (v.nx + tw - 1) / tw;
            p.inv_d[q] = 1.0f / (float)p.tiles_x[q];
            tiles += p.tiles_x[q] * ((v.ny + th - 1) / th);
        }
    }
    p.tile_begin[n] = tiles;
    if (FLAV == FLAV_VECTOR)
        k_step_group_vec<S, ODD, GMODE, MAXL><<<tiles, BATCH_THREADS, 0, st>>>(p);
    else
        k_step_group<S, ODD, FLAV == FLAV_GENERAL, GMODE, MAXL><<<tiles, BATCH_THREADS, 0, st>>>(p);
    return cudaGetLastError();
}

template <typename S, bool ODD, int FLAV, int GMODE>
static cudaError_t launch_group_sized(const State* const* m, const int* cur, const int* l2tw,
                                      int n, cudaStream_t st) {
    for (int q0 = 0; q0 < n; q0 += 64) {
        const int c = n - q0 < 64 ? n - q0 : 64;
        const cudaError_t e = c <= 4
            ? launch_group<S, ODD, FLAV, GMODE, 4>(m + q0, cur + q0, l2tw + q0, c, st)
            : launch_group<S, ODD, FLAV, GMODE, 64>(m + q0, cur + q0, l2tw + q0, c, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename S, bool ODD, int FLAV>
static cudaError_t launch_group_g(const State* const* m, const int* cur, const int* l2tw, int n,
                                  int g_mode, cudaStream_t st) {
    return g_mode == G_OFF ? launch_group_sized<S, ODD, FLAV, G_OFF>(m, cur, l2tw, n, st)
                           : launch_group_sized<S, ODD, FLAV, G_LAGGED>(m, cur, l2tw, n, st);
}

template <typename S>
cudaError_t Ops<S>::step_group(const State* const* m, const int* cur, const int* l2tw, int n,
                               bool odd, int flavour, int g_mode, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (odd) {
        if (flavour == FLAV_GENERAL) return launch_group_g<S, true, FLAV_GENERAL>(m, cur, l2tw, n, g_mode, st);
        if (flavour == FLAV_VECTOR) return launch_group_g<S, true, FLAV_VECTOR>(m, cur, l2tw, n, g_mode, st);
        return launch_group_g<S, true, FLAV_PERIODIC>(m, cur, l2tw, n, g_mode, st);
    }
    if (flavour == FLAV_GENERAL) return launch_group_g<S, false, FLAV_GENERAL>(m, cur, l2tw, n, g_mode, st);
    if (flavour == FLAV_VECTOR) return launch_group_g<S, false, FLAV_VECTOR>(m, cur, l2tw, n, g_mode, st);
    return launch_group_g<S, false, FLAV_PERIODIC>(m, cur, l2tw, n, g_mode, st);
}

template <typename S>
cudaError_t Ops<S>::ghost_pass(const State& s, int k, cudaStream_t st) {
    if (s.nghost <= 0) return cudaSuccess;
    using C = typename Fmt<S>::C;
    State v = s;
    v.parity = s.parity ^ (k & 1);
    if (s.g_mode == G_LAGGED) v.cur = s.cur ^ (k & 1);
    const Args<C> a = make_args<C>(v);
    const int t = 128, g = (s.nghost + t - 1) / t;
    if (v.parity == 0) k_ghosts<S, true><<<g, t, 0, st>>>(a, s.ghosts, s.nghost);
    else k_ghosts<S, false><<<g, t, 0, st>>>(a, s.ghosts, s.nghost);
    return cudaGetLastError();
}

}  // namespace trt
