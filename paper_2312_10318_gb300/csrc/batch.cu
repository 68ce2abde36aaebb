// Batches: several lattices advanced together.  Per time step the members are
// grouped by (storage format, boundary flavour, G mode, parity of the current
// level) and each group is one specialised launch (lb_batch.cuh); runs of
// kGraphSteps steps are captured once into a CUDA graph and replayed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "lb_batch.cuh"
#include "lb_handle.h"

namespace {

constexpr int kGraphSteps = 32;  // steps per captured graph (even: parity and Phi
                                 // buffers return to their start after a replay)

}  // namespace

struct trtrlb_batch {
    cudaStream_t stream = nullptr;
    cudaStream_t copy_in = nullptr;    // uploads, downloads, and initial states and
    cudaStream_t copy_out = nullptr;   // moments, of trtrlb_batch_solve (created on
    cudaStream_t aux = nullptr;        // its first call)
    std::vector<trtrlb_t> lats;
    cudaGraphExec_t graph = nullptr;
    std::vector<int> graph_sig;   // (parity, cur) of every member when captured
    char err[256] = "";
};

namespace {

int fail(trtrlb_batch* b, int code, const char* msg) {
    std::snprintf(b->err, sizeof b->err, "%s", msg);
    return code;
}

int cuda_fail(trtrlb_batch* b, cudaError_t e, const char* where) {
    std::snprintf(b->err, sizeof b->err, "%s: %s", where, cudaGetErrorString(e));
    return TRTRLB_ECUDA;
}

void drop_graph(trtrlb_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_sig.clear();
}

std::vector<int> signature(const trtrlb_batch* b) {
    std::vector<int> sig;
    for (const trtrlb_lattice* h : b->lats) {
        sig.push_back(h->s.parity);
        sig.push_back(h->s.cur);
        sig.push_back(h->s.f == h->f ? 0 : 1);   // two-buffer lattices alternate buffers
    }
    return sig;
}

int log2i(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

#define TRT_DISPATCH_S(storage, CALL)                                                 \
    [&]() -> cudaError_t {                                                            \
        switch (storage) {                                                            \
            case TRTRLB_F64: { using S = double; return trt::Ops<S>::CALL; }          \
            case TRTRLB_F64_DW: { using S = trt::f64dw; return trt::Ops<S>::CALL; }   \
            case TRTRLB_F32: { using S = float; return trt::Ops<S>::CALL; }           \
            case TRTRLB_F16_SHIFTED: { using S = __half; return trt::Ops<S>::CALL; }  \
            default: { using S = __nv_bfloat16; return trt::Ops<S>::CALL; }           \
        }                                                                             \
    }()

// Launches n steps of every member, starting from the members' current
// states; step q sees parity ^ (q & 1) and, for lagged G, cur ^ (q & 1).
cudaError_t launch_steps(trtrlb_batch* b, int64_t n) {
    using Key = std::tuple<int, int, int, int>;  // storage, flavour, g_mode, odd
    for (int64_t q = 0; q < n; ++q) {
        const int flip = (int)(q & 1);
        std::map<Key, std::vector<int>> groups;
        for (int i = 0; i < (int)b->lats.size(); ++i) {
            const trtrlb_lattice* h = b->lats[i];
            if (h->s.g_mode == TRTRLB_G_CURRENT) continue;   // two-buffer kernel, below
            const int flav = h->s.general ? trt::FLAV_GENERAL : (h->s.vec ? trt::FLAV_VECTOR : trt::FLAV_PERIODIC);
            groups[Key{h->p.storage, flav, h->s.g_mode, h->s.parity ^ flip}].push_back(i);
        }
        for (const auto& kv : groups) {
            const Key& k = kv.first;
            std::vector<const trt::State*> m;
            std::vector<int> cur, l2;
            for (int i : kv.second) {
                const trtrlb_lattice* h = b->lats[i];
                m.push_back(&h->s);
                cur.push_back(h->s.g_mode == TRTRLB_G_LAGGED ? (h->s.cur ^ flip) : h->s.cur);
                l2.push_back(log2i(h->tile_w));
            }
            const cudaError_t e = TRT_DISPATCH_S(
                std::get<0>(k), step_group(m.data(), cur.data(), l2.data(), (int)m.size(),
                                           std::get<3>(k) != 0, std::get<1>(k),
                                           std::get<2>(k), b->stream));
            if (e != cudaSuccess) return e;
        }
        // two-buffer (G_CURRENT) members: the small TMA-fed ones share
        // launches, the others run one launch each
        std::vector<const trt::State*> tma;
        for (trtrlb_lattice* h : b->lats)
            if (shares_tma_launch(h)) tma.push_back(&h->s);
        if (!tma.empty()) {
            const cudaError_t e = trt::Ops<float>::step_ab_group(tma.data(), (int)tma.size(), flip, b->stream);
            if (e != cudaSuccess) return e;
        }
        for (trtrlb_lattice* h : b->lats) {
            if (h->s.g_mode == TRTRLB_G_CURRENT) {
                if (shares_tma_launch(h)) continue;
                const cudaError_t e = TRT_DISPATCH_S(h->p.storage, step_ab(h->s, flip, b->stream));
                if (e != cudaSuccess) return e;
                continue;
            }
            if (h->s.nghost == 0) continue;
            const cudaError_t e = TRT_DISPATCH_S(h->p.storage, ghost_pass(h->s, flip, b->stream));
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

int capture(trtrlb_batch* b) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(b, e, "graph capture");
    const cudaError_t le = launch_steps(b, kGraphSteps);
    e = cudaStreamEndCapture(b->stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(b, le, "graph capture launch");
    }
    if (e != cudaSuccess) return cuda_fail(b, e, "graph capture end");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return cuda_fail(b, e, "graph instantiate");
    }
    b->graph_sig = signature(b);
    return TRTRLB_OK;
}

}  // namespace

extern "C" {

int trtrlb_batch_create(void* stream, trtrlb_batch_t* out) {
    if (!out) return TRTRLB_EINVAL;
    trtrlb_batch* b = new (std::nothrow) trtrlb_batch();
    if (!b) return TRTRLB_ENOMEM;
    b->stream = static_cast<cudaStream_t>(stream);
    *out = b;
    return TRTRLB_OK;
}

int trtrlb_batch_destroy(trtrlb_batch_t b) {
    if (!b) return TRTRLB_OK;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    if (b->copy_in) cudaStreamDestroy(b->copy_in);
    if (b->copy_out) cudaStreamDestroy(b->copy_out);
    if (b->aux) cudaStreamDestroy(b->aux);
    delete b;
    return TRTRLB_OK;
}

int trtrlb_batch_set(trtrlb_batch_t b, const trtrlb_t* lattices, int count) {
    if (!b) return TRTRLB_EINVAL;
    b->err[0] = 0;
    if (count < 0 || (count > 0 && !lattices)) return fail(b, TRTRLB_EINVAL, "bad lattice list");
    std::vector<trtrlb_t> l(lattices, lattices + count);
    for (int q = 0; q < count; ++q) {
        if (!l[q]) return fail(b, TRTRLB_EINVAL, "null lattice in the list");
        for (int r = 0; r < q; ++r)
            if (l[r] == l[q]) return fail(b, TRTRLB_EINVAL, "a lattice appears twice");
    }
    drop_graph(b);
    b->lats.swap(l);
    return TRTRLB_OK;
}

int trtrlb_batch_solve(trtrlb_batch_t b, const double* const* rho, const double* const* ux,
                       const double* const* uy, int64_t nsteps, double* const* rho_out,
                       double* const* ux_out, double* const* uy_out) {
    if (!b) return TRTRLB_EINVAL;
    b->err[0] = 0;
    cudaError_t e = cudaSuccess;
    if (!b->copy_in) e = cudaStreamCreateWithFlags(&b->copy_in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !b->copy_out) e = cudaStreamCreateWithFlags(&b->copy_out, cudaStreamNonBlocking);
    if (e == cudaSuccess && !b->aux) {
        // the highest priority: its short, compute-bound kernels are scheduled
        // between the steps' blocks instead of after them
        int lo = 0, hi = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->aux, cudaStreamNonBlocking, hi);
    }
    if (e != cudaSuccess) return cuda_fail(b, e, "solve streams");
    return trt::solve_members(b->lats.data(), (int)b->lats.size(), b->stream, b->aux, b->copy_in, b->copy_out,
                              rho, ux, uy, nsteps, rho_out, ux_out, uy_out, b->err);
}

int trtrlb_batch_step(trtrlb_batch_t b, int64_t nsteps) {
    if (!b) return TRTRLB_EINVAL;
    b->err[0] = 0;
    if (nsteps < 0) return fail(b, TRTRLB_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0 || b->lats.empty()) return TRTRLB_OK;
    int64_t done = 0;
    if (b->stream != nullptr && nsteps >= kGraphSteps) {
        if (b->graph && b->graph_sig != signature(b)) drop_graph(b);
        if (!b->graph) {
            if (int rc = capture(b)) return rc;
        }
        for (; done + kGraphSteps <= nsteps; done += kGraphSteps) {
            const cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) return cuda_fail(b, e, "graph launch");
        }
    }
    const cudaError_t e = launch_steps(b, nsteps - done);
    if (e != cudaSuccess) return cuda_fail(b, e, "batch step");
    for (trtrlb_lattice* h : b->lats) {
        if (h->s.g_mode == TRTRLB_G_CURRENT) {
            if (nsteps & 1) {
                void* t = h->s.f;
                h->s.f = h->s.f2;
                h->s.f2 = t;
            }
        } else {
            h->s.parity ^= (int)(nsteps & 1);
            if (h->s.g_mode == TRTRLB_G_LAGGED) h->s.cur ^= (int)(nsteps & 1);
        }
        h->t += nsteps;
    }
    return TRTRLB_OK;
}

const char* trtrlb_batch_last_error(trtrlb_batch_t b) { return b ? b->err : ""; }

}  // extern "C"
