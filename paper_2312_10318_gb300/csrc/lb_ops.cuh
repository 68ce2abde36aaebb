// Host-side launchers of the device kernels, one instantiation per storage
// format (lb_ops_<fmt>.cu), so the formats compile in parallel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace trt {

// Storage tag of FP64 populations with double-word FP32 arithmetic (lb_dw.cuh).
struct f64dw;

// Threads per block of the diagnostics reduction.
constexpr int DIAG_THREADS = 256;

// Kernel flavours of a lattice's step.
enum : int { FLAV_GENERAL = 0, FLAV_PERIODIC = 1, FLAV_VECTOR = 2 };

// Nodes per thread of the vectorised kernel: 16 bytes of FP64 / FP32
// storage, VEC16_NODES elements of 16-bit storage.
constexpr int VEC16_NODES = 4;
inline int vec_width(int storage_bytes) { return storage_bytes == 2 ? VEC16_NODES : 16 / storage_bytes; }

// Format-independent description of a lattice's device state.
// TMA-fed two-buffer kernel (lb_ab_tma.cuh): a tile of 32 x TMA_TH nodes, a
// thread owning TMA_TH / 8 of them (one per 8 rows), and its box x0-4 .. x0+35
// by y0-1 .. y0+TMA_TH, all 9 population planes, in one of TMA_STAGES
// shared-memory stages.
constexpr int TMA_TH = 8, TMA_STAGES = 2;
constexpr int TMA_BX = 40, TMA_BY = TMA_TH + 2, TMA_XOFF = 4;
// Polls of an mbarrier before a kernel's wait gives up (microseconds suffice
// for a tile copy; the limit only bounds a wait that would never end).
constexpr long long kDefaultWaitLimit = 1ll << 22;

struct State {
    void* f;              // populations, S[9][ny][pitch]
    void* f2;             // second buffer of the two-buffer G_CURRENT kernel (else null)
    void* phi[2];         // Phi buffers, C[2][ny][pitch]
    int cur;              // phi[cur] holds the previous level
    const uint8_t* mask;  // device [ny][pitch] or nullptr
    const uint8_t* seg;   // general lattices: device [ny][segs], 1 where the 32-node row
                          // segment and all its neighbours are plain fluid (or nullptr)
    int segs;             // segments per row, (nx + 31) / 32
    const int* ghosts;    // device list of outlet ghost offsets
    int nghost;
    int nx, ny, pitch;
    long long plane;
    int px, py;
    bool general;         // walls, mask or non-periodic edges present
    bool vec;             // the vectorised kernel runs this lattice
    int col_h;            // G_CURRENT: rows per band of the column-walking two-buffer
                          // kernel, which runs the step; 0: another kernel
    int tile_w;           // scalar kernels: block of tile_w x (256 / tile_w) nodes
    int g_mode;
    double tau1, tau2, gx, gy, rho0;
    double wall_ux, wall_uy, wall_rho;
    double outlet_rho;    // density of Zou-He pressure outlet nodes
    int parity;           // parity of the current level
    // FP32 periodic G_CURRENT lattices: TMA descriptors (CUtensorMap, host
    // memory) of the population buffers, tma_map[k] describing tma_buf[k]
    const void* tma_buf[2];
    const void* tma_map[2];
    int tma_grid;         // persistent grid of the TMA kernel (0: not used)
    int* kerr;            // device flag: a kernel's bounded wait ran out
    long long wait_limit; // polls before a kernel's wait gives up
};

template <typename S> struct Ops {
    // One time step (plus the outlet-ghost pass); flips parity and Phi buffers.
    static cudaError_t step(State& s, cudaStream_t st);
    static cudaError_t phi_static(State& s, cudaStream_t st);
    static cudaError_t init(State& s, const double* rho, const double* ux, const double* uy,
                            cudaStream_t st);
    static cudaError_t moments(const State& s, double* rho, double* ux, double* uy,
                               cudaStream_t st);
    static cudaError_t get_f(const State& s, double* f, double* phi, cudaStream_t st);
    static cudaError_t set_f(State& s, const double* f, const double* phi, cudaStream_t st);
    // Deterministic FP64 diagnostics; part holds diag_blocks() * 8 doubles.
    static cudaError_t diagnostics(const State& s, double* part, double* out, cudaStream_t st);
    // One batched step of n lattices that share the kernel flavour (FLAV_*),
    // G mode and the parity of their current level (odd); cur[q] is the Phi
    // buffer holding member q's previous level, log2_tw[q] its tile width
    // (scalar flavours).  Launches ceil(n / 64) kernels.
    static cudaError_t step_group(const State* const* members, const int* cur, const int* log2_tw,
                                  int n, bool odd, int flavour, int g_mode, cudaStream_t st);
    // Outlet-ghost pass after step index k of a sequence that started at the
    // state's current parity and Phi buffer.
    static cudaError_t ghost_pass(const State& s, int k, cudaStream_t st);
    // Two-buffer G_CURRENT step q of a sequence starting from s.f (the buffers
    // alternate with q); the caller swaps s.f / s.f2 after an odd count.
    static cudaError_t step_ab(const State& s, int q, cudaStream_t st);
    // Persistent grid (resident CTAs per SM x SMs) of the TMA-fed two-buffer
    // kernel on the current device; 0 for formats that do not have it.
    static int tma_grid();
    // Whether the TMA-fed two-buffer kernel advances this lattice (FP32,
    // periodic without a mask, G_CURRENT, descriptors present).
    static bool tma_eligible(const State& s);
    // Two-buffer step q of n such lattices, up to 16 per launch.
    static cudaError_t step_ab_group(const State* const* members, int n, int q, cudaStream_t st);
};

int diag_blocks(const State& s);

// FP64 comparison of velocity fields (compare.cu): blocks of the first level
// (as many as diag_blocks gives for the same node count) and the launcher.
// ux, uy, rx, ry are dense [ny][nx] device fields; mask is a lattice's pitched
// device mask or null; part holds compare_blocks(nx * ny) * 8 doubles; out
// receives TRTRLB_CMP_N doubles (include/trtrlb.h).
int compare_blocks(long long nodes);
cudaError_t compare_fields(const double* ux, const double* uy, const double* rx, const double* ry,
                           const uint8_t* mask, int nx, int ny, int pitch, int px, int py,
                           double* part, double* out, cudaStream_t st);

}  // namespace trt
