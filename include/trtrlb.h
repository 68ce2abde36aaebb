/*
 * trtrlb — GB300-native D2Q9 two-relaxation-time regularized lattice
 * Boltzmann (TRT-RLB) library: the C ABI.
 *
 * The scheme is the one of Yu, Qin, Chen, Shu and Yuan (arXiv 2312.10318).
 * Equation names below are that paper's equation labels (eq2, eq4, eq6, eq9,
 * eq11, eq_Gi, eq_a20, eq_a29, eq_mu ...).  One time step is eq2: collide with
 * the regularized TRT operator, add the cubic-error compensation G_i (eq_Gi)
 * and the forcing term F_i (eq6), stream, and apply half-way bounce-back
 * (eq_a20) at walls.
 *
 * Conventions shared by every entry point:
 *   - Lattice units: dx = dt = c = 1, c_s^2 = 1/3.
 *   - A field is nx*ny values, index y*nx + x (x fastest).  Populations are
 *     9*nx*ny values, index (i*ny + y)*nx + x, with the paper's D2Q9 numbering
 *     e_0..e_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1).
 *   - Pointers to fields may be host or device memory (detected per call).
 *     The caller owns them; the library copies in and out.
 *   - Every call is asynchronous on the handle's stream, except where a call
 *     writes into host memory: that call synchronises the stream before it
 *     returns.
 *   - Return value: TRTRLB_OK (0) or a negative TRTRLB_E* code; on error the
 *     handle is left as it was, and trtrlb_last_error() describes the cause.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef TRTRLB_H
#define TRTRLB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define TRTRLB_OK 0
#define TRTRLB_EINVAL (-1)    /* invalid argument or parameter combination      */
#define TRTRLB_ENOMEM (-2)    /* device or host allocation failed               */
#define TRTRLB_ECUDA (-3)     /* a CUDA runtime call failed                     */
#define TRTRLB_EUNSTABLE (-4) /* diagnostics found NaN/Inf or |u| beyond bound   */
#define TRTRLB_ETIMEOUT (-5)  /* a bounded wait gave up                         */
#define TRTRLB_ENOTSUP (-6)   /* combination not built into this library        */

/* Population storage formats.  All collision arithmetic of the reduced
 * formats runs in FP32 on the shifted deviation f_i - w_i rho0; FP64 storage
 * runs FP64 arithmetic.  F64_DW is a 64-bit double-word format: each
 * population is a pair of FP32 numbers hi + lo (~48 significant bits) and the
 * collision runs in double-word FP32 arithmetic, which GB300 executes several
 * times faster than its FP64 pipe; results agree with FP64 to ~1e-13. */
#define TRTRLB_F64 0
#define TRTRLB_F32 1
#define TRTRLB_F16_SHIFTED 2
#define TRTRLB_BF16_SHIFTED 3
#define TRTRLB_F64_DW 4

/* Time level of Phi_abg = rho u_a^3 delta... in the compensation term G_i
 * (eq_Gi).  The paper does not say which level; d_gamma Phi is a central
 * difference over neighbouring nodes.
 *   LAGGED : Phi from the previous step (Phi^{-1} := Phi^0), used by the
 *            in-place AA kernels, which cannot see neighbours' current moments.
 *   CURRENT: Phi of the current step, by the two-buffer kernel (Phi of each
 *            tile and its halo computed in shared memory; twice the
 *            population memory, no Phi traffic).
 *   OFF    : G_i = 0. */
#define TRTRLB_G_LAGGED 0
#define TRTRLB_G_CURRENT 1
#define TRTRLB_G_OFF 2

/* Boundary mask classes (one byte per node). */
#define TRTRLB_FLUID 0
#define TRTRLB_SOLID 1  /* stationary wall node: half-way bounce-back, eq_a20 */
#define TRTRLB_INLET 2  /* moving wall node (velocity inlet): bounce-back with
                           the correction -2 w_i rho_w (e_i.u_w)/c_s^2      */
#define TRTRLB_OUTLET 3 /* zero-gradient outlet ghost: does not collide and
                           re-emits the post-collision populations of its
                           inward neighbour (x-1, y), which must be fluid    */
#define TRTRLB_PRESSURE 4 /* Zou-He constant-pressure outlet (Sec. III D): a
                           node on the last column x = nx-1 of a lattice not
                           periodic in x; it collides like a fluid node after
                           the populations entering across the edge (e_x < 0)
                           are rebuilt so that rho = outlet_rho, u_y = 0 and
                           the normal non-equilibrium parts bounce back.
                           Links leaving across the edge are open; Phi beyond
                           the edge is the node's own.  Every read of the
                           state (step, moments, populations, diagnostics)
                           sees the rebuilt values.                          */
#define TRTRLB_HALO 5   /* halo node of a sub-lattice (trtrlb_slabs_*): stands
                           for a fluid node another sub-lattice updates; it
                           does not collide, links into it stream, and its
                           populations and Phi are written by the exchange  */
#define TRTRLB_HALO_PRESSURE 6 /* halo node standing for a TRTRLB_PRESSURE node
                           another sub-lattice updates: as TRTRLB_HALO, and a
                           Phi taken from its populations (G_CURRENT) takes
                           the Zou-He rebuild first, as the owner's does    */

/* Problem statement (Sec. II B, eq2; eq_mu; eq_a2; eq_a29). */
typedef struct {
    int32_t nx, ny;          /* lattice size: 1 <= ny <= 131070, 1 <= nx <= 2^24,
                                (nx + 63) * ny <= 2^30                           */
    int32_t periodic_x;      /* 1: periodic in x; 0: stationary half-way walls   */
    int32_t periodic_y;      /*    just outside x = -1/2 and x = nx - 1/2 (y alike) */
    double tau_s;            /* tau_{s,1} > 1/2: relaxes the 1st and 2nd order;
                                kinematic viscosity nu = (tau_s - 1/2)/3 (eq_mu) */
    double tau_s2;           /* tau_{s,2} >= 1/2: relaxes the 3rd order, or NaN  */
    double magic;            /* Lambda_s = (tau_s - 1/2)(tau_s2 - 1/2) (eq_a29),
                                or NaN.  Exactly one of tau_s2 / magic may be NaN;
                                if both are given they must agree to 1e-12 rel. */
    double gx, gy;           /* body acceleration; F = rho g (eq_a2)             */
    double rho0;             /* reference density of the shifted storage (> 0)   */
    double wall_ux, wall_uy; /* velocity of TRTRLB_INLET nodes                   */
    double wall_rho;         /* density rho_w in the moving-wall correction      */
    double outlet_rho;       /* density of TRTRLB_PRESSURE nodes (> 0)           */
    int32_t storage;         /* TRTRLB_F64 | F32 | F16_SHIFTED | BF16_SHIFTED | F64_DW */
    int32_t g_mode;          /* TRTRLB_G_LAGGED | G_CURRENT | G_OFF              */
} trtrlb_params;

typedef struct trtrlb_lattice* trtrlb_t;

/* Fills *p with defaults: periodic 64x64, tau_s = 0.8, magic = 1/4 (tau_s2 NaN),
 * no force, rho0 = wall_rho = outlet_rho = 1, FP32 storage, LAGGED. */
void trtrlb_default_params(trtrlb_params* p);

/* Creates a lattice and allocates its device memory on the current device.
 *   mask   : NULL (all fluid) or nx*ny bytes of TRTRLB_* classes, host memory;
 *   stream : cudaStream_t all work of the handle is ordered on (NULL = legacy
 *            default stream);
 *   out    : receives the handle; unchanged on error.
 * The populations start at rest with density rho0.  Errors: EINVAL (bad size,
 * tau, magic/tau_s2, storage, mask class, outlet without a fluid inward
 * neighbour, pressure outlet off the last column or on a lattice periodic in
 * x), ENOMEM, ECUDA. */
int trtrlb_create(const trtrlb_params* p, const uint8_t* mask, void* stream, trtrlb_t* out);

/* Frees all memory of the handle (synchronises its stream).  NULL is a no-op. */
int trtrlb_destroy(trtrlb_t h);

/* Changes the stream later work is ordered on.  Work already queued on the
 * old stream is not waited for: the caller orders the two streams (an event
 * recorded on the old one and waited for on the new one). */
int trtrlb_set_stream(trtrlb_t h, void* stream);

/* Initial state from macroscopic fields (t = 0):
 *   f_i = f_i^eq(rho, u) - (1/2) w_i e_i.F / c_s^2   (eq4, eq11),
 * and Phi of the previous level := Phi of (rho, u).  rho may be NULL (rho0
 * everywhere); ux, uy are required.  Values at non-fluid nodes are ignored. */
int trtrlb_init(trtrlb_t h, const double* rho, const double* ux, const double* uy);

/* Advances nsteps >= 0 time steps of eq2 (asynchronous). */
int trtrlb_step(trtrlb_t h, int64_t nsteps);

/* Macroscopic fields of the current state (eq11): rho = sum f_i and
 * u = (sum e_i f_i)/rho + g/2, FP64.  Any pointer may be NULL.  Non-fluid
 * nodes report 0. */
int trtrlb_moments(trtrlb_t h, double* rho, double* ux, double* uy);

/* Populations f_i(x, t) of the current state as 9*nx*ny FP64 values, and
 * optionally (phi != NULL) the previous-level Phi as 2*nx*ny values
 * (Phi_xxx then Phi_yyy; LAGGED only, zeros otherwise).  Non-fluid nodes
 * report 0 populations. */
int trtrlb_get_f(trtrlb_t h, double* f, double* phi);

/* Replaces the populations of the current state (9*nx*ny FP64 values, rounded
 * to the storage format).  phi == NULL: the previous-level Phi becomes that of
 * the new state; otherwise 2*nx*ny values are taken as given.  Values at
 * non-fluid nodes are ignored. */
int trtrlb_set_f(trtrlb_t h, const double* f, const double* phi);

/* Number of steps taken since the last init / set_f. */
int64_t trtrlb_time(trtrlb_t h);

/* FP64 diagnostics over the fluid nodes of the current state (deterministic
 * fixed-order reduction).  out[8] receives:
 *   [0] total mass sum rho, [1] sum rho u_x, [2] sum rho u_y,
 *   [3] kinetic energy sum rho |u|^2 / 2, [4] max |u|,
 *   [5] number of nodes whose populations are not finite,
 *   [6], [7] momentum-exchange force on the walls (Sec. III D) x, y:
 *   the sum over links from fluid nodes into solid nodes or across
 *   non-periodic edges of 2 e_i f_ibar(x_f, t).
 * out may be host or device memory. */
int trtrlb_diagnostics(trtrlb_t h, double* out);

/* Comparison of velocity fields in FP64 on the device, for the error norms of
 * Sec. III: the relative L2 error of eq_n1, the largest local change that the
 * steady-state test of eq_n2 divides by the characteristic speed, and the same
 * relative L2 error of the vorticity.  The sums run over the fluid nodes of h
 * (and pressure outlet nodes) in a fixed order, so the same fields always give
 * the same bits.  The vorticity omega = d_x u_y - d_y u_x is taken by central
 * differences on the node lattice at the fluid nodes whose four axis
 * neighbours are fluid nodes of the domain (wrapped across periodic edges).
 * out receives TRTRLB_CMP_N doubles:
 *   [0] sqrt(sum |u - u_ref|^2 / sum |u_ref|^2)            (eq_n1 for u)
 *   [1] max |u - u_ref|                                      (eq_n2 numerator)
 *   [2] sqrt(sum (omega - omega_ref)^2 / sum omega_ref^2)    (eq_n1 for omega)
 *   [3] sqrt(sum |u - u_ref|^2 / nodes)                      (RMS difference)
 *   [4] sum |u - u_ref|^2, [5] sum |u_ref|^2,
 *   [6] sum (omega - omega_ref)^2, [7] sum omega_ref^2,
 *   [8] nodes compared, [9] nodes skipped because u or u_ref is not finite.
 * A ratio with a zero denominator is 0 when its numerator is 0, else +inf.
 * out may be host (the call then synchronises) or device memory. */
#define TRTRLB_CMP_N 10

/* u of h's current state (eq11, as trtrlb_moments gives it) against the
 * reference fields ux_ref, uy_ref ([ny][nx] FP64, host or device; values at
 * non-fluid nodes are ignored). */
int trtrlb_compare(trtrlb_t h, const double* ux_ref, const double* uy_ref, double* out);

/* u of a's current state against u of b's (the reference): same nx and ny;
 * the nodes compared are a's fluid nodes.  The work runs on a's stream after
 * the work queued so far on b's stream, and b's later work waits for it. */
int trtrlb_compare_lattices(trtrlb_t a, trtrlb_t b, double* out);

/* The same eight diagnostics as trtrlb_diagnostics, for a state given in the
 * canonical layout, computed without allocating any memory.  The paper has no
 * counterpart.  It is for callers that cannot call cudaMalloc when they need
 * the numbers: a host application that hands this library only memory carved
 * from its own pool under a fixed device budget, or a latency-critical loop
 * that must not take the implicit synchronisation of an allocation.
 *   f      : device, 9*nx*ny FP64 populations (layout above; e.g. what
 *            trtrlb_get_f writes), read only;
 *   mask   : device, nx*ny bytes of TRTRLB_* classes, or NULL (all fluid);
 *            pressure outlet nodes count as fluid with f taken as given (a
 *            state from trtrlb_get_f already holds the rebuilt values);
 *   periodic_x/y, gx, gy : as in trtrlb_params (u includes the g/2 shift);
 *   out    : device, 8 doubles, same meaning as in trtrlb_diagnostics;
 *   stream : cudaStream_t the two kernels run on (asynchronous).
 * The reduction's partial sums live in one static device array of 512 KiB
 * (8 doubles for each of at most 8192 blocks of 2048 nodes) that every GPU
 * loading the library holds until the process exits.  Lattices of more than
 * 16,777,216 nodes (4096^2) are rejected with TRTRLB_EINVAL, as are null or
 * host pointers.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress, with that device current) and caches it for the life
 * of the process: make that first call before any stream capture, and do not
 * call this entry point on a device after cudaDeviceReset has been called on
 * it (the cached address no longer names the array).  All calls share the
 * array: calls that overlap on the GPU (on different streams, or on several
 * host threads) race and corrupt each other's results; serialise them.
 * Nothing needs clearing between calls: every call overwrites the partial
 * sums it reads. */
int trtrlb_diagnostics_noalloc(const double* f, const uint8_t* mask, int32_t nx, int32_t ny,
                               int32_t periodic_x, int32_t periodic_y, double gx, double gy,
                               double* out, void* stream);

/* Measured FP64 arithmetic ceiling of the current device (the paper has no
 * counterpart): the throughput of independent chains of double-precision
 * fused multiply-adds (2 flops each) over about `seconds` (at least 10 ms),
 * timed with CUDA events on `stream` (cudaStream_t, NULL = legacy), written to
 * *tflops in TFLOP/s.  FP64-storage steps, which GB300's FP64 pipe bounds long
 * before HBM does, are reported against it.  Synchronises the stream.
 * EINVAL for a null output or a non-positive duration, ECUDA on a CUDA error. */
int trtrlb_fp64_fma_rate(void* stream, double seconds, double* tflops);

/* Kernel shape of a lattice's step (the autotuner's knobs; results do not
 * depend on them).  variant: TRTRLB_KERNEL_AUTO (the vector kernel where it
 * applies for FP32/FP16/BF16, the scalar one for FP64 and F64_DW; with
 * G_CURRENT on a periodic lattice without a mask the TMA-fed kernel for FP32
 * and the column kernel for FP64/FP16/BF16 where its bands give at least
 * half as many warps as the device holds resident -- on 152 SMs from 1024^2
 * nodes for FP16/BF16 and 512^2 for FP64 --, the plain one below),
 * TRTRLB_KERNEL_SCALAR (one node per thread; for G_CURRENT the plain
 * two-buffer kernel instead of the TMA-fed one), TRTRLB_KERNEL_VECTOR
 * (a vector of nodes per thread: 2 for FP64, 4 otherwise; ENOTSUP unless the
 * lattice is periodic in both directions, has no mask and nx is a multiple
 * of that width).
 * TRTRLB_KERNEL_COLUMN (G_CURRENT only: the two-buffer kernel whose warps walk
 * down bands of rows of 30 columns, keeping the Phi of the rows above and
 * below in registers; bands of 32, 16 or 8 rows (FP64: 16, 8 or 4), the
 * tallest that fills the device; ENOTSUP unless the lattice is periodic in
 * both directions, has no mask and stores FP64, FP32, FP16 or BF16).
 * tile_w: width in nodes of the scalar kernel's 256-thread tile (32, 64, 128
 * or 256; 0 keeps the current one). */
#define TRTRLB_KERNEL_AUTO 0
#define TRTRLB_KERNEL_SCALAR 1
#define TRTRLB_KERNEL_VECTOR 2
#define TRTRLB_KERNEL_COLUMN 3
int trtrlb_set_kernel(trtrlb_t h, int32_t variant, int32_t tile_w);

/* Checkpoint and resume (the paper has none): the raw device state -- the
 * populations as stored (format, AA level and layout), both Phi buffers, the
 * level's parity, the Phi buffer index and the step count -- as an opaque
 * image of trtrlb_state_bytes(h) bytes in host or device memory.  Loading it
 * into a lattice created with the same parameters and mask continues bit for
 * bit as the saved one would have (trtrlb_get_f / trtrlb_set_f go through
 * FP64 and the shift by w_i rho0, which rounds for FP64 storage).  Both
 * synchronise the handle's stream.  trtrlb_load returns EINVAL for an image of
 * another size, format or G mode. */
int64_t trtrlb_state_bytes(trtrlb_t h);
int trtrlb_save(trtrlb_t h, void* image);
int trtrlb_load(trtrlb_t h, const void* image);

/* Bounded waits.  The TMA-fed G_CURRENT kernel (FP32, periodic, no mask)
 * waits on an mbarrier for each tile copy; after `polls` unsuccessful polls
 * (default 4,194,304: far beyond a copy's microseconds) it records the failure,
 * drains its copies in flight and returns, and the next trtrlb_moments /
 * trtrlb_get_f / trtrlb_diagnostics with host outputs reports TRTRLB_ETIMEOUT
 * (the state of that step is then undefined).  polls = 0 makes every such wait
 * give up at once, to exercise that path. */
int trtrlb_set_wait_limit(trtrlb_t h, int64_t polls);

/* The kernel in use: *vector = 1 for the vector kernel; *tile_w as above.
 * Either pointer may be NULL. */
int trtrlb_get_kernel(trtrlb_t h, int32_t* vector, int32_t* tile_w);

/* Which step kernel the lattice's current settings select (format, G mode,
 * boundaries, size and trtrlb_set_kernel), as *kind:
 *   TRTRLB_STEP_AA            fused AA stream-collide, one node per thread
 *                             (k_step; in a batch k_step_group)
 *   TRTRLB_STEP_AA_VECTOR     the same, a vector of nodes per thread
 *   TRTRLB_STEP_AB            two-buffer step with Phi at the current level,
 *                             one node per thread
 *   TRTRLB_STEP_AB_TMA        two-buffer step fed by TMA, one launch for this
 *                             lattice, in a batch too
 *   TRTRLB_STEP_AB_TMA_SHARED the same kernel; in a batch it shares launches
 *                             (up to 16 lattices each) with the other such
 *                             members
 *   TRTRLB_STEP_AB_COLUMN     two-buffer step walking columns.
 * Host only, no device work.  EINVAL for a null handle or output. */
#define TRTRLB_STEP_AA 0
#define TRTRLB_STEP_AA_VECTOR 1
#define TRTRLB_STEP_AB 2
#define TRTRLB_STEP_AB_TMA 3
#define TRTRLB_STEP_AB_TMA_SHARED 4
#define TRTRLB_STEP_AB_COLUMN 5
int trtrlb_step_kernel(trtrlb_t h, int32_t* kind);

/* ---- slab decomposition -----------------------------------------------------
 * One lattice split into nslabs sub-lattices of consecutive rows (y), the
 * single-device form of a multi-GPU domain split (the paper has none; its
 * scheme is node-local apart from streaming and d Phi, so a split needs only a
 * one-row halo).  Slab k owns rows [row0_k, row0_k + rows_k) (rows as even as
 * possible, the first ny % nslabs slabs one more) and is a lattice handle of
 * its own, with a TRTRLB_HALO row on each side that faces another slab (both
 * sides when the lattice is periodic in y).  Every step exchanges rows with
 * device copies on the slabs' stream: before it, the previous level's
 * Phi_yyy of the boundary rows (LAGGED); around a step from an odd level of
 * the in-place pattern, the y-moving populations of the boundary rows (in
 * before, out after); around a two-buffer step (G_CURRENT), all nine
 * populations of the boundary rows before it (the halo's Phi is then taken at
 * the current level from them) and the populations pushed into the halo rows
 * after it.  Results equal the undivided lattice's bit for bit (G_CURRENT in
 * FP32 against its plain two-buffer kernel: the TMA-fed one contracts into FMAs
 * differently).  Masks with outlet ghosts (or halo nodes) give ENOTSUP; host or
 * device pointers are accepted where fields are passed (global [ny][nx] /
 * [9][ny][nx] layouts); calls synchronise except step. */
typedef struct trtrlb_slabs* trtrlb_slabs_t;
int trtrlb_slabs_create(const trtrlb_params* p, const uint8_t* mask, int32_t nslabs, void* stream,
                        trtrlb_slabs_t* out);
int trtrlb_slabs_destroy(trtrlb_slabs_t s);
int trtrlb_slabs_init(trtrlb_slabs_t s, const double* rho, const double* ux, const double* uy);
int trtrlb_slabs_step(trtrlb_slabs_t s, int64_t nsteps);
int trtrlb_slabs_get_f(trtrlb_slabs_t s, double* f);
int trtrlb_slabs_moments(trtrlb_slabs_t s, double* rho, double* ux, double* uy);
/* Sums (mass, momenta, energy, non-finite count, wall force) and the maximum
 * speed over the slabs' owned nodes; out: 8 doubles, host or device. */
int trtrlb_slabs_diagnostics(trtrlb_slabs_t s, double* out);
/* Number of slabs; slab k's handle, first owned global row, owned rows and
 * whether it has a halo row below (its owned rows then start at local row 1).
 * The handles stay owned by s. */
int32_t trtrlb_slabs_count(trtrlb_slabs_t s);
int trtrlb_slabs_slab(trtrlb_slabs_t s, int32_t k, trtrlb_t* h, int32_t* row0, int32_t* rows,
                      int32_t* halo_below);
const char* trtrlb_slabs_last_error(trtrlb_slabs_t s);

/* ---- batches ---------------------------------------------------------------
 * A batch advances several lattices together: per time step one kernel launch
 * per storage format covers every tile of every lattice in the batch (the
 * same per-node update as trtrlb_step, so results are those of stepping each
 * lattice alone).  G_CURRENT members take the two-buffer kernel: FP32 periodic
 * ones without a mask share its TMA-fed launches (up to 16 lattices each; the
 * results equal the single-lattice launch's up to the compiler's FMA
 * contraction, a few FP32 ulps), the others take one launch each.  Runs of 32
 * or more steps replay a captured CUDA graph when
 * the batch's stream is not the legacy default stream.  Lattices keep their
 * own parity and step count; all of them must live on the batch's device and
 * their other work must be ordered with the batch's stream by the caller
 * (simplest: create them on the same stream).  A lattice must stay alive while
 * it is a member; call trtrlb_batch_set again before destroying it. */
typedef struct trtrlb_batch* trtrlb_batch_t;

/* Creates an empty batch ordered on `stream` (cudaStream_t; NULL = legacy). */
int trtrlb_batch_create(void* stream, trtrlb_batch_t* out);

/* Replaces the members (count >= 0 distinct handles).  EINVAL on a null or
 * repeated handle.  Invalidates the captured graph. */
int trtrlb_batch_set(trtrlb_batch_t b, const trtrlb_t* lattices, int count);

/* Advances every member by nsteps >= 0 steps (asynchronous). */
int trtrlb_batch_step(trtrlb_batch_t b, int64_t nsteps);

/* End-to-end solve of every member: member k starts from the fields
 * (rho[k], ux[k], uy[k]) as trtrlb_init does (eq11 moments; rho[k], or the
 * array rho itself, NULL for rho0), advances nsteps >= 0 time steps, and its
 * eq11 moments are written to rho_out[k], ux_out[k], uy_out[k] (each, or each
 * array, may be NULL).  Arrays are [ny][nx] doubles in host or device memory;
 * host arrays should be page-locked for the copies to run beside the steps.
 * The members advance one after another, each with its own launches (as
 * trtrlb_step), so that the upload of the next member and the download of
 * the previous one run on two copy streams of the batch while a member
 * steps, and the next member's initial state and the previous one's moments
 * on a fourth stream; the results equal trtrlb_init, trtrlb_step and
 * trtrlb_moments of each member alone.  Ordered after the work already queued on the members'
 * streams and on the batch's stream; returns when the outputs are written.
 * EINVAL for a bad argument, ECUDA for a CUDA error, ETIMEOUT as
 * trtrlb_moments. */
int trtrlb_batch_solve(trtrlb_batch_t b, const double* const* rho, const double* const* ux,
                       const double* const* uy, int64_t nsteps, double* const* rho_out,
                       double* const* ux_out, double* const* uy_out);

/* Frees the batch (not its lattices); synchronises its stream. */
int trtrlb_batch_destroy(trtrlb_batch_t b);

/* Message of the batch's last error ("" if none). */
const char* trtrlb_batch_last_error(trtrlb_batch_t b);

/* Device bytes held by the handle. */
int64_t trtrlb_device_bytes(trtrlb_t h);

/* Static description of an error code. */
const char* trtrlb_strerror(int code);

/* Message of the last error on this handle ("" if none); NULL handle: the
 * last error of a failed trtrlb_create on this thread. */
const char* trtrlb_last_error(trtrlb_t h);

#ifdef __cplusplus
}
#endif
#endif /* TRTRLB_H */
