// 128-bit vectorised AA step for periodic lattices without a mask.
//
// Each thread owns V consecutive nodes of one row (FP64 2, FP32 4: 16 bytes;
// FP16/BF16 4: 8 bytes) and moves every population with one aligned vector
// load and one aligned vector store.  A warp owns 32 V consecutive nodes of
// a row.  Even steps touch only the nodes' own slots.  On odd steps the slots
// of the x-neighbours are shifted by one element: a thread loads the aligned
// vector at its own x0 and takes the missing element from the neighbouring
// lane with a warp shuffle; only the first lane of a warp segment, the last
// one, and the lanes at the ends of a row go to memory for that element
// (scalar accesses, with periodic wrap).  Stores are realigned the same way:
// a lane stores the full aligned vector when both lanes next to it belong to
// the same row segment, and otherwise writes the elements it owns one by one.
// Requires nx % V == 0 and pitch % V == 0.
#pragma once
#include "lb_device.cuh"
#include "lb_ops.cuh"

namespace trt {

// ---- packed vectors -----------------------------------------------------------
// P: the register pack of V elements;
// shift_up(A, w) = [w.last, A[0], ..., A[V-2]] where w is the lane-neighbour's
// last word; shift_down(A, w) = [A[1], ..., A[V-1], w.first].
template <typename S> struct Pk;

template <> struct Pk<float> {
    using P = float4;
    // elements 2k and 2k + 1 as compute values, and back
    static __device__ __forceinline__ void unpack2(const P& p, int k, float& a, float& b) {
        a = k == 0 ? p.x : p.z;
        b = k == 0 ? p.y : p.w;
    }
    static __device__ __forceinline__ void pack2(P& p, int k, float a, float b) {
        if (k == 0) { p.x = a; p.y = b; } else { p.z = a; p.w = b; }
    }
    using W = float;  // one shuffle word
    static constexpr int V = 4;
    static __device__ __forceinline__ float get(const P& p, int v) {
        return v == 0 ? p.x : (v == 1 ? p.y : (v == 2 ? p.z : p.w));
    }
    static __device__ __forceinline__ void set(P& p, int v, float c) {
        if (v == 0) p.x = c; else if (v == 1) p.y = c; else if (v == 2) p.z = c; else p.w = c;
    }
    static __device__ __forceinline__ W last_word(const P& p) { return p.w; }
    static __device__ __forceinline__ W first_word(const P& p) { return p.x; }
    static __device__ __forceinline__ W word_of(float s) { return s; }  // edge element as a word
    static __device__ __forceinline__ P shift_up(const P& a, W prev) { return make_float4(prev, a.x, a.y, a.z); }
    static __device__ __forceinline__ P shift_down(const P& a, W next) { return make_float4(a.y, a.z, a.w, next); }
    static __device__ __forceinline__ float elem(const P& p, int v) { return get(p, v); }  // raw storage element
};

template <> struct Pk<double> {
    using P = double2;
    static __device__ __forceinline__ void unpack2(const P& p, int, double& a, double& b) {
        a = p.x;
        b = p.y;
    }
    static __device__ __forceinline__ void pack2(P& p, int, double a, double b) {
        p.x = a;
        p.y = b;
    }
    using W = double;
    static constexpr int V = 2;
    static __device__ __forceinline__ double get(const P& p, int v) { return v == 0 ? p.x : p.y; }
    static __device__ __forceinline__ void set(P& p, int v, double c) {
        if (v == 0) p.x = c; else p.y = c;
    }
    static __device__ __forceinline__ W last_word(const P& p) { return p.y; }
    static __device__ __forceinline__ W first_word(const P& p) { return p.x; }
    static __device__ __forceinline__ W word_of(double s) { return s; }
    static __device__ __forceinline__ P shift_up(const P& a, W prev) { return make_double2(prev, a.x); }
    static __device__ __forceinline__ P shift_down(const P& a, W next) { return make_double2(a.y, next); }
    static __device__ __forceinline__ double elem(const P& p, int v) { return get(p, v); }
};

// 8 x 16-bit elements in four 32-bit words; element 2k is the low half of
// word k, element 2k + 1 the high half.
template <typename H> struct Cvt2;
template <> struct Cvt2<__half> {
    static __device__ __forceinline__ float2 to_float2(unsigned int w) {
        return __half22float2(*reinterpret_cast<const __half2*>(&w));
    }
    static __device__ __forceinline__ unsigned int from_floats(float a, float b) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const unsigned int*>(&h);
    }
};
template <> struct Cvt2<__nv_bfloat16> {
    static __device__ __forceinline__ float2 to_float2(unsigned int w) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
    }
    static __device__ __forceinline__ unsigned int from_floats(float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const unsigned int*>(&h);
    }
};

template <int NW> struct Words;
template <> struct Words<2> {
    using P = uint2;
    static __device__ __forceinline__ unsigned int get(const P& p, int k) { return k == 0 ? p.x : p.y; }
    static __device__ __forceinline__ void set(P& p, int k, unsigned int w) {
        if (k == 0) p.x = w; else p.y = w;
    }
};
template <> struct Words<4> {
    using P = uint4;
    static __device__ __forceinline__ unsigned int get(const P& p, int k) {
        return k == 0 ? p.x : (k == 1 ? p.y : (k == 2 ? p.z : p.w));
    }
    static __device__ __forceinline__ void set(P& p, int k, unsigned int w) {
        if (k == 0) p.x = w; else if (k == 1) p.y = w; else if (k == 2) p.z = w; else p.w = w;
    }
};

// Double-word storage: packs of two (hi, lo) pairs in one float4.
template <> struct Pk<f64dw> {
    using P = float4;
    using W = df64;
    static constexpr int V = 2;
    static __device__ __forceinline__ df64 get(const P& p, int v) {
        return v == 0 ? df64(p.x, p.y) : df64(p.z, p.w);
    }
    static __device__ __forceinline__ void unpack2(const P& p, int, df64& a, df64& b) {
        a = df64(p.x, p.y);
        b = df64(p.z, p.w);
    }
    static __device__ __forceinline__ void pack2(P& p, int, df64 a, df64 b) {
        p = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
    static __device__ __forceinline__ W last_word(const P& p) { return df64(p.z, p.w); }
    static __device__ __forceinline__ W first_word(const P& p) { return df64(p.x, p.y); }
    static __device__ __forceinline__ W word_of(f64dw s) { return df64(s.hi, s.lo); }
    static __device__ __forceinline__ P shift_up(const P& a, W prev) {
        return make_float4(prev.hi, prev.lo, a.x, a.y);
    }
    static __device__ __forceinline__ P shift_down(const P& a, W next) {
        return make_float4(a.z, a.w, next.hi, next.lo);
    }
    static __device__ __forceinline__ f64dw elem(const P& p, int v) {
        return v == 0 ? f64dw{p.x, p.y} : f64dw{p.z, p.w};
    }
};

// 2 NW x 16-bit elements in NW 32-bit words (element 2k: low half of word k).
template <typename H, int NW> struct Pk16 {
    using WD = Words<NW>;
    using P = typename WD::P;
    using W = unsigned int;
    static constexpr int V = 2 * NW;
    static __device__ __forceinline__ unsigned int word(const P& p, int k) { return WD::get(p, k); }
    static __device__ __forceinline__ void set_word(P& p, int k, unsigned int w) { WD::set(p, k, w); }
    static __device__ __forceinline__ void unpack2(const P& p, int k, float& a, float& b) {
        const float2 f = Cvt2<H>::to_float2(word(p, k));
        a = f.x;
        b = f.y;
    }
    static __device__ __forceinline__ void pack2(P& p, int k, float a, float b) {
        set_word(p, k, Cvt2<H>::from_floats(a, b));
    }
    static __device__ __forceinline__ unsigned short bits(const P& p, int v) {
        const unsigned int w = word(p, v >> 1);
        return (unsigned short)((v & 1) ? (w >> 16) : (w & 0xffffu));
    }
    static __device__ __forceinline__ W last_word(const P& p) { return word(p, NW - 1); }
    static __device__ __forceinline__ W first_word(const P& p) { return word(p, 0); }
    // an edge element loaded from memory, placed where shift_up / shift_down
    // expect it (high half for prev, low half for next: both are filled)
    static __device__ __forceinline__ W word_of(H s) {
        const unsigned int b = *reinterpret_cast<const unsigned short*>(&s);
        return (b << 16) | b;
    }
    static __device__ __forceinline__ P shift_up(const P& a, W prev) {
        P r;
#pragma unroll
        for (int k = 0; k < NW; ++k)
            set_word(r, k, __byte_perm(k == 0 ? prev : word(a, k - 1), word(a, k), 0x5432));
        return r;
    }
    static __device__ __forceinline__ P shift_down(const P& a, W next) {
        P r;
#pragma unroll
        for (int k = 0; k < NW; ++k)
            set_word(r, k, __byte_perm(word(a, k), k == NW - 1 ? next : word(a, k + 1), 0x5432));
        return r;
    }
    static __device__ __forceinline__ H elem(const P& p, int v) {
        const unsigned short b = bits(p, v);
        return *reinterpret_cast<const H*>(&b);
    }
};
// 16-bit formats run VEC16_NODES nodes per thread (8-byte vectors): measured
// faster than 16-byte vectors, whose register footprint halves the resident
// warps of this latency-sensitive kernel.
template <> struct Pk<__half> : Pk16<__half, VEC16_NODES / 2> {};
template <> struct Pk<__nv_bfloat16> : Pk16<__nv_bfloat16, VEC16_NODES / 2> {};

// aligned vector load / store of one pack (16 or 8 bytes)
template <typename S>
__device__ __forceinline__ typename Pk<S>::P ld16(const S* p) {
    return *reinterpret_cast<const typename Pk<S>::P*>(p);
}
template <typename S>
__device__ __forceinline__ void st16(S* p, const typename Pk<S>::P& v) {
    *reinterpret_cast<typename Pk<S>::P*>(p) = v;
}

template <typename W>
__device__ __forceinline__ W shfl_up1(W w) { return __shfl_up_sync(0xffffffffu, w, 1); }
template <typename W>
__device__ __forceinline__ W shfl_down1(W w) { return __shfl_down_sync(0xffffffffu, w, 1); }
template <>
__device__ __forceinline__ df64 shfl_up1<df64>(df64 w) {
    return df64(__shfl_up_sync(0xffffffffu, w.hi, 1), __shfl_up_sync(0xffffffffu, w.lo, 1));
}
template <>
__device__ __forceinline__ df64 shfl_down1<df64>(df64 w) {
    return df64(__shfl_down_sync(0xffffffffu, w.hi, 1), __shfl_down_sync(0xffffffffu, w.lo, 1));
}

// Element I of a pack written to memory (storage format).
template <typename S>
__device__ __forceinline__ S pack_elem(const typename Pk<S>::P& p, int v) {
    return (S)Pk<S>::elem(p, v);
}

// Elements 1 .. V-1 of a pack to p[1 .. V-1], and elements 0 .. V-2 to
// p[0 .. V-2] (p = a row + x0, x0 a multiple of V, so p is aligned to the
// pack): for V = 4 the aligned pair of the four goes in one access.
template <typename S>
__device__ __forceinline__ void store_from1(S* p, const typename Pk<S>::P& w) {
    constexpr int V = Pk<S>::V;
    if constexpr (V == 4 && sizeof(S) == 2) {
        p[1] = pack_elem<S>(w, 1);
        *reinterpret_cast<unsigned int*>(p + 2) = Pk<S>::word(w, 1);
    } else if constexpr (V == 4 && std::is_same<S, float>::value) {
        p[1] = w.y;
        *reinterpret_cast<float2*>(p + 2) = make_float2(w.z, w.w);
    } else {
#pragma unroll
        for (int v = 1; v < V; ++v) p[v] = pack_elem<S>(w, v);
    }
}
template <typename S>
__device__ __forceinline__ void store_to_last(S* p, const typename Pk<S>::P& w) {
    constexpr int V = Pk<S>::V;
    if constexpr (V == 4 && sizeof(S) == 2) {
        *reinterpret_cast<unsigned int*>(p) = Pk<S>::word(w, 0);
        p[2] = pack_elem<S>(w, 2);
    } else if constexpr (V == 4 && std::is_same<S, float>::value) {
        *reinterpret_cast<float2*>(p) = make_float2(w.x, w.y);
        p[2] = w.z;
    } else {
#pragma unroll
        for (int v = 0; v < V - 1; ++v) p[v] = pack_elem<S>(w, v);
    }
}

// ---- the vectorised node-segment update ---------------------------------------
// Lane `lane` of a warp owns nodes x0 .. x0 + V - 1 of row y (active when
// x0 < nx).  All 32 lanes must call this together (warp shuffles).
template <typename S, bool ODD, int GMODE>
__device__ __forceinline__ void seg_step(const Args<typename Fmt<S>::C>& a, int x0, int y,
                                         int lane) {
    using C = typename Fmt<S>::C;
    using K = Pk<S>;
    using P = typename K::P;
    constexpr int V = K::V;
    S* __restrict__ F = static_cast<S*>(a.f);
    const bool active = x0 < a.nx;
    const int ym = y == 0 ? a.ny - 1 : y - 1;
    const int yp = y == a.ny - 1 ? 0 : y + 1;
    const int xl = x0 == 0 ? a.nx - 1 : x0 - 1;        // element left of the vector
    const int xr = x0 + V == a.nx ? 0 : x0 + V;         // element right of the vector
    const bool edge_l = lane == 0 || x0 == 0;           // no active left lane in this segment
    const bool edge_r = lane == 31 || x0 + V == a.nx;   // no active right lane in this segment
    const long long rowy = (long long)y * a.pitch;

    // ---- lagged Phi: d_x Phi_xxx and d_y Phi_yyy (first: fewer live registers)
    C dpx[V], dpy[V];
    if (GMODE == G_LAGGED) {
        const C* Px = a.phi_in + rowy;
        const C* Pym = a.phi_in + a.plane + (long long)ym * a.pitch;
        const C* Pyp = a.phi_in + a.plane + (long long)yp * a.pitch;
        C px[V], pm[V], pp[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            px[v] = active ? Px[x0 + v] : C(0);
            pm[v] = active ? Pym[x0 + v] : C(0);
            pp[v] = active ? Pyp[x0 + v] : C(0);
        }
        C left = shfl_up1(px[V - 1]);
        C right = shfl_down1(px[0]);
        if (edge_l && active) left = Px[xl];
        if (edge_r && active) right = Px[xr];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const C l = v == 0 ? left : px[v - 1];
            const C r = v == V - 1 ? right : px[v + 1];
            dpx[v] = C(0.5) * (r - l);
            dpy[v] = C(0.5) * (pp[v] - pm[v]);
        }
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) dpx[v] = dpy[v] = C(0);
    }

    // ---- gather the nine populations --------------------------------------
    P d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if (!ODD) {
            d[i] = active ? ld16<S>(F + (long long)i * a.plane + rowy + x0) : P{};
        } else {
            const int dx = ex(i), dy = ey(i);
            const int r = dy > 0 ? ym : (dy < 0 ? yp : y);     // row of x - e_i
            const long long base = (long long)opp(i) * a.plane + (long long)r * a.pitch;
            const P A = active ? ld16<S>(F + base + x0) : P{};
            if (dx == 0) {
                d[i] = A;
            } else if (dx > 0) {   // source x - 1
                typename K::W w = shfl_up1(K::last_word(A));
                if (edge_l && active) w = K::word_of(F[base + xl]);
                d[i] = K::shift_up(A, w);
            } else {               // source x + 1
                typename K::W w = shfl_down1(K::first_word(A));
                if (edge_r && active) w = K::word_of(F[base + xr]);
                d[i] = K::shift_down(A, w);
            }
        }
    }

    // ---- collide every node of the vector, two at a time ----------------------
    P o[9];
    C phx[V], phy[V];
#pragma unroll
    for (int k = 0; k < V / 2; ++k) {
        C lo[9], hi[9], olo[9], ohi[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) K::unpack2(d[i], k, lo[i], hi[i]);
        collide<C>(lo, dpx[2 * k], dpy[2 * k], a.k1, a.k1lo, a.k2, a.k2lo, a.kf, a.gx, a.gy, a.rho0, olo,
                   phx[2 * k], phy[2 * k]);
        collide<C>(hi, dpx[2 * k + 1], dpy[2 * k + 1], a.k1, a.k1lo, a.k2, a.k2lo, a.kf, a.gx, a.gy, a.rho0, ohi,
                   phx[2 * k + 1], phy[2 * k + 1]);
#pragma unroll
        for (int i = 0; i < 9; ++i) K::pack2(o[i], k, olo[i], ohi[i]);
    }
    if (GMODE == G_LAGGED && active) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            a.phi_out[rowy + x0 + v] = phx[v];
            a.phi_out[a.plane + rowy + x0 + v] = phy[v];
        }
    }

    // ---- scatter --------------------------------------------------------------
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if (!ODD) {
            if (active) st16<S>(F + (long long)opp(i) * a.plane + rowy + x0, o[i]);
        } else {
            const int dx = ex(i), dy = ey(i);
            const int r = dy > 0 ? yp : (dy < 0 ? ym : y);     // row of x + e_i
            S* base = F + (long long)i * a.plane + (long long)r * a.pitch;
            if (dx == 0) {
                if (active) st16<S>(base + x0, o[i]);
            } else if (dx > 0) {   // targets x0 + 1 .. x0 + V
                const P Wv = K::shift_up(o[i], shfl_up1(K::last_word(o[i])));
                if (active) {
                    if (!edge_l) st16<S>(base + x0, Wv);
                    else store_from1<S>(base + x0, Wv);
                    if (edge_r) base[xr] = pack_elem<S>(o[i], V - 1);
                }
            } else {               // targets x0 - 1 .. x0 + V - 2
                const P Wv = K::shift_down(o[i], shfl_down1(K::first_word(o[i])));
                if (active) {
                    if (!edge_r) st16<S>(base + x0, Wv);
                    else store_to_last<S>(base + x0, Wv);
                    if (edge_l) base[xl] = pack_elem<S>(o[i], 0);
                }
            }
        }
    }
}

// Single-lattice launch: block of 256 threads = 8 warps, warp w of block b
// owns segment s = 8 b + w of the (row, segment) list.
template <typename S, bool ODD, int GMODE>
__global__ void __launch_bounds__(256, sizeof(S) == 2 ? 4 : 3) k_step_vec(Args<typename Fmt<S>::C> a, int segs_per_row) {
    constexpr int V = Pk<S>::V;
    const int lane = (int)threadIdx.x & 31;
    const long long s = (long long)blockIdx.x * 8 + ((int)threadIdx.x >> 5);
    const long long nseg = (long long)segs_per_row * a.ny;
    if (s >= nseg) return;   // whole warp leaves together
    const int y = (int)(s / segs_per_row);
    const int x0 = (int)(s % segs_per_row) * 32 * V + lane * V;
    seg_step<S, ODD, GMODE>(a, x0, y, lane);
}

}  // namespace trt
