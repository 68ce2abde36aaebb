// Internal layout of a lattice handle, shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "lb_ops.cuh"
#include "trtrlb.h"

struct trtrlb_lattice {
    trtrlb_params p;
    trt::State s;
    cudaStream_t stream;
    int64_t t;           // steps since init / set_f
    void* f;             // device allocations owned by the handle
    void* f2;            // second population buffer (G_CURRENT only)
    void* phi;           // both Phi buffers in one allocation
    uint8_t* mask;
    uint8_t* seg;        // interior row segments of a general lattice (State::seg), or null
    int* ghosts;
    double* stage;       // FP64 staging for host transfers and comparisons
    int stage_fields;    // its size in fields of nx * ny doubles (3, 4 or 11)
    double* part;        // diagnostics partials (scratch)
    double* dout;        // result of diagnostics (8 doubles) and comparisons (TRTRLB_CMP_N)
    int64_t bytes;
    int tile_w;          // scalar-kernel tile width in the batched path (32 .. 256 nodes)
    int variant;         // TRTRLB_KERNEL_AUTO / SCALAR / VECTOR
    void* tmaps;         // two CUtensorMap (host) of the FP32 periodic G_CURRENT kernel, or null
    int* kerr;           // device flag set when a kernel's bounded wait ran out, or null
    int tma_grid;        // persistent grid of the TMA kernel on this device (0: none)
    int sms;             // multiprocessors of the handle's device
    char err[256];
};

// Lattices below this many nodes share the TMA-fed two-buffer launches of a
// batch (one persistent grid, one tail: 3 x 1024^2 FP32 54.2 -> 56.6 GLUPS);
// larger ones take a launch each (one 4096^2 lattice steps alone in 0.231 ms,
// three of them sharing a launch in 0.90 ms).
constexpr long long kTmaShareMaxNodes = 2048ll * 2048ll;

inline bool shares_tma_launch(const trtrlb_lattice* h) {
    return h->s.g_mode == TRTRLB_G_CURRENT && h->p.storage == TRTRLB_F32 &&
           trt::Ops<float>::tma_eligible(h->s) && (long long)h->p.nx * h->p.ny < kTmaShareMaxNodes;
}

namespace trt {
// Body of trtrlb_batch_solve over the members m[0 .. count): see trtrlb.h.
// st runs the members' steps, aux their initial states and moments; cin and
// cout their uploads and downloads.
int solve_members(trtrlb_lattice* const* m, int count, cudaStream_t st, cudaStream_t aux, cudaStream_t cin,
                  cudaStream_t cout, const double* const* rho, const double* const* ux, const double* const* uy,
                  int64_t nsteps, double* const* rho_out, double* const* ux_out, double* const* uy_out,
                  char* err);
}  // namespace trt
