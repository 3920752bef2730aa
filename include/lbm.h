/*
 * lbm.h - C ABI of the GB300 library for the three-population phase-field lattice-Boltzmann
 * method of Zhan, Liang, Chai & Shi, "Phase-field-based lattice Boltzmann method for the
 * transport of insoluble surfactant in two-phase flows" (arXiv 2408.15654).
 *
 * One time step advances, on one 2-D D2Q9 grid, three coupled populations:
 *   f -> phi   conservative Allen-Cahn phase field                  (Sec. 3.1)
 *   g -> psi   interface-confined surfactant (Jain's equation)     (Sec. 3.2)
 *   h -> u, P  consistent incompressible flow with the capillary and
 *              Marangoni forces of the surfactant EOS sigma(psi)    (Sec. 3.3, Sec. 2.3)
 * with moment-space MRT collision (Sec. 4) and streaming, periodic in x, periodic or bounded by
 * half-way bounce-back walls in y.  Every step runs in hand-written sm_103a CUDA kernels; there
 * is no CPU fallback.
 *
 * Conventions shared by all calls
 *   - Lattice units: dx = dt = c = 1, cs^2 = 1/3.  Cells sit at integer (x, y), 0 <= x < nx,
 *     0 <= y < ny.  Walls (bc_y = LBM_BC_WALLS) lie half a cell below row 0 and above row ny-1.
 *   - Host fields are row-major double arrays of ny * nx values, index y * nx + x.
 *   - Every call returns an int status: LBM_OK (0) or one of the LBM_E* codes below.  No C++
 *     exception crosses the ABI.  lbm_last_error() gives a message for the calling thread.
 *   - All device work is enqueued on the CUDA stream given to lbm_create.  Calls marked
 *     "synchronous" wait for that stream before returning.
 *   - A handle is not thread safe; use one handle per host thread or serialise the calls.
 */
#ifndef GB300_LBM_H
#define GB300_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define LBM_OK 0
#define LBM_EINVAL 1    /* invalid argument or unsupported parameter combination            */
#define LBM_ENOMEM 2    /* workspace too small                                               */
#define LBM_ECUDA 3     /* a CUDA runtime call failed (message in lbm_last_error)            */
#define LBM_EUNSTABLE 4 /* the device flagged a non-finite value, |u| >= 0.3, or psi >= 1
                           under the Langmuir EOS (sticky until the next lbm_init_fields)    */
#define LBM_ETIMEOUT 5  /* a bounded device wait gave up                                     */
#define LBM_ESTATE 6    /* call out of order (e.g. lbm_step before lbm_init_fields)          */

/* ---- enumerations ---------------------------------------------------------------------- */
#define LBM_BC_PERIODIC 0   /* periodic in y (x is always periodic)                          */
#define LBM_BC_WALLS 1      /* half-way bounce-back walls below row 0 and above row ny-1      */

#define LBM_EOS_LINEAR 0    /* sigma = sigma0 (1 - E0 psi)            (Sec. 2.3, linear EOS)  */
#define LBM_EOS_LANGMUIR 1  /* sigma = sigma0 [1 + E0 ln(1 - psi)]    (Sec. 2.3, Langmuir EOS) */

#define LBM_STORE_FP32 0    /* populations stored as float                                   */
#define LBM_STORE_FP16 1    /* as FP16 deviations from references (see lbm_workspace_bytes) */
#define LBM_STORE_BF16 2    /* as BF16 deviations from references                            */
#define LBM_STORE_FP16_FG 3 /* f and g as FP16 deviations, h as float                        */
#define LBM_STORE_BF16_FG 4 /* f and g as BF16 deviations, h as float                        */

#define LBM_VELOCITY_SOLVED 0     /* u from the flow populations h (Sec. 3.3)                  */
#define LBM_VELOCITY_PRESCRIBED 1 /* u imposed (the ux, uy given to lbm_init_fields, constant in
                                     time); only f and g are stored and advanced, P is 0, the EOS
                                     and the flow parameters are unused (the convection test of
                                     Sec. 4)                                                   */

#define LBM_MEM_HOST 0      /* pointer arguments are host memory (pageable or pinned; pinned
                               arrays are read and written by the kernels directly, pageable
                               ones are staged in device memory)                              */
#define LBM_MEM_DEVICE 1    /* pointer arguments are device memory on the handle's device    */

#define LBM_PHI 1u          /* moment masks for lbm_get_moments                              */
#define LBM_PSI 2u
#define LBM_UX 4u
#define LBM_UY 8u
#define LBM_P 16u

#define LBM_SUM_PHI 0       /* lbm_reduce selectors                                          */
#define LBM_SUM_PSI 1

/* ---- parameters (plain data, copied by lbm_create) --------------------------------------
 * Physical constants in lattice units.  The relaxation rates s_f, s_g, s_h are (s0..s4) of the
 * diagonal S = diag(s0, s1, s1, s2, s2, s2, s3, s3, s4) (Sec. 4); the transport entries are
 * recomputed by the library and ignored here:
 *   1/s1^f = M_phi/cs2 + 1/2,  1/s1^g = D/cs2 + 1/2 (Eq. for s1^g),  1/s2^h = mu/(rho cs2) + 1/2.
 * A value s_h[4] <= 0 means s4^h = s2^h (recommended: keeps plane Couette flow exact).
 * Requirements: nx >= 2, ny >= 2, phiA != phiB, W > 0, M_phi > 0, D > 0, rhoA, rhoB > 0,
 * muA, muB > 0, all rates in (0, 2) (s_h[4] may be <= 0), storage one of LBM_STORE_*.
 * With rhoA != rhoB the step includes the mass flux S, the grad rho terms of H, m2H and P and
 * the time derivative of S (Sec. 2.3, 3.3); the workspace then holds a mass-flux history too.  */
typedef struct lbm_params {
    int32_t nx, ny;         /* grid size                                                     */
    int32_t bc_y;           /* LBM_BC_PERIODIC or LBM_BC_WALLS                               */
    int32_t eos;            /* LBM_EOS_LINEAR or LBM_EOS_LANGMUIR                            */
    int32_t storage;        /* one of LBM_STORE_* (arithmetic is FP32 in every mode)         */
    int32_t velocity;       /* LBM_VELOCITY_SOLVED or LBM_VELOCITY_PRESCRIBED                */
    double u_top, u_bot;    /* x velocity of the top and bottom wall (LBM_BC_WALLS)          */
    double phiA, phiB;      /* order parameter of the pure phases (Sec. 2.1)                 */
    double rhoA, rhoB;      /* densities (Sec. 2.3, linear in phi)                           */
    double muA, muB;        /* dynamic viscosities (Sec. 2.3, linear in phi)                 */
    double W;               /* interface width (Sec. 2.1)                                    */
    double M_phi;           /* phase-field mobility (Sec. 2.1)                               */
    double D;               /* surfactant diffusivity (Sec. 2.2)                             */
    double sigma0, E0;      /* clean-interface tension and elasticity number (Sec. 2.3)      */
    double gx, gy;          /* body-force acceleration, F_b = rho g                          */
    double n_eps;           /* n = grad phi/|grad phi| if |grad phi| > n_eps, else n = 0     */
    double s_f[5], s_g[5], s_h[5];
} lbm_params;

typedef struct lbm_handle lbm_handle;

/* Bytes of device workspace lbm_create needs for these parameters: two population buffers, two
 * velocity-history buffers, a status word and the reduction partials.  Returns LBM_EINVAL for bad
 * parameters (among them a grid outside nx, ny >= 2, nx * ny <= 2^30, ny <= 524280).
 * Layout: the workspace starts with the two population buffers, each the larger of
 * B * (ny + 4) * pitch and 40 * nx * ny bytes (a buffer that is not current stages the five FP64
 * fields of host transfers) rounded up to a multiple of 256, with pitch = nx + 10 rounded up to a
 * multiple of 32 and
 * B = 104 (FP32 storage), 52 (FP16, BF16) or 68 (FP16_FG, BF16_FG); with
 * LBM_VELOCITY_PRESCRIBED, 72 (FP32) or 36 (16-bit).  A buffer holds 9 planes of (f_i, g_i)
 * pairs followed by 4 planes of (h_1, h_2), (h_3, h_4), (h_5, h_6), (h_7, h_8) pairs (h_0 never
 * influences the step; no h planes with a prescribed velocity), each plane ny + 4 rows of pitch
 * cells: cell (x, y) is at row y + 2,
 * column x + 8, inside a ghost frame of copies (periodic images; bounce-back values in the rows
 * next to walls) that the library maintains.  After lbm_init_fields and k steps the current
 * state is buffer k mod 2 (buffer 0 at offset 0).
 * FP32 storage holds the values.  16-bit storage (FP16 / BF16, arithmetic still FP32) holds
 * each value divided by its lattice weight w_i, as a scaled deviation from a reference (the
 * _FG modes store only f and g this way and h as FP32 values):
 * (f_i / w_i - phi_ref) S_f and (g_i / w_i) S_g with phi_ref = (phiA + phiB)/2, and
 * (h_i / w_i - 3 rho c_i.u) S_h with u the velocity that the cell holding the slot wrote to the
 * velocity history in the same step; S = (1, 256, 4096) for FP16 and 1 for BF16.  Dividing by
 * w_i makes the bulk equilibria exactly representable; removing 3 rho c_i.u keeps the pressure
 * part of h (about 1e-5) above the 16-bit rounding of the velocity part (about 1e-3).  Steps
 * store 16-bit values with stochastic rounding, its random bits a hash of the cell index and
 * the step count (so a run is deterministic and a restored state continues bit for bit).  The
 * velocity history (two buffers of (ny + 4) x pitch float pairs in the same frame, alternating
 * like the populations) follows the population buffers; with rhoA != rhoB (and a solved flow) two
 * more such buffers hold the mass flux S of the last step. */
int lbm_workspace_bytes(const lbm_params* p, size_t* bytes);

/* Create a handle on the current CUDA device.
 *   d_workspace: device memory of at least lbm_workspace_bytes bytes, 256-byte aligned, owned
 *                by the caller, kept alive until lbm_destroy (the library never frees it).
 *   cuda_stream: cudaStream_t on which all work of this handle is enqueued (NULL = legacy
 *                default stream).
 *   out:         receives the handle (host memory owned by the library).
 * The handle holds no state until lbm_init_fields. */
int lbm_create(const lbm_params* p, void* d_workspace, size_t bytes, void* cuda_stream,
               lbm_handle** out);

/* Set all populations to the equilibria of the given fields (f_eq of Sec. 3.1, g_eq of Sec. 3.2,
 * h_eq of Sec. 3.3 with S = 0) and clear the status word and the time-derivative history (the
 * first step after this call uses zero time derivatives).  Each pointer is a row-major array of
 * ny * nx doubles in `mem` (LBM_MEM_HOST or LBM_MEM_DEVICE); all five are required.
 * Values are checked for finiteness (and psi < 1 under the Langmuir EOS) on the device.
 * Synchronous: the caller may free or reuse the arrays when it returns. */
int lbm_init_fields(lbm_handle* h, const double* phi, const double* psi, const double* ux,
                    const double* uy, const double* P, int mem);

/* Advance n >= 0 time steps: one fused collide-stream kernel launch per step (pull streaming,
 * stencils on halo tiles in shared memory, moment-space collision of f, g and h).
 * Asynchronous: errors found by the device surface at the next synchronous call. */
int lbm_step(lbm_handle* h, int64_t n);

/* Macroscopic fields at the current time level (phi = sum f, psi = sum g, u from
 * rho u = sum c h + F/2, P from the pressure equation of Sec. 3.3).  For every bit set in mask
 * (LBM_PHI, LBM_PSI, LBM_UX, LBM_UY, LBM_P, in that order of out[0..4]) out[k] must point to ny * nx
 * doubles in `mem`.  Synchronous.  Returns LBM_EUNSTABLE if the status word is set. */
int lbm_get_moments(lbm_handle* h, unsigned mask, double* const out[5], int mem);

/* Sum over the grid of phi (LBM_SUM_PHI) or psi (LBM_SUM_PSI) in FP64: each cell's populations
 * are summed in FP64 by warp shuffles, then blocks, then one final block (deterministic order).
 * Both sums are conserved by the method (sum F_i = sum G_i = 0).  Before the first step after
 * lbm_init_fields the populations are staged where the first step pulls them (next to a wall, in
 * the wall's ghost row), and the sum is taken over the values each cell pulls; afterwards over
 * each cell's own post-collision values.  *out is host memory.  Synchronous. */
int lbm_reduce(lbm_handle* h, int what, double* out);

/* Failure-detection self-test.  Launches one warp on cuda_stream that waits, with the bounded
 * wait every step kernel uses for its copies, on an mbarrier that nothing completes.  The wait
 * gives up after at most about one second and records a timeout in d_word (a device pointer to 4
 * bytes owned by the caller), without faulting: the context stays usable.  Synchronous.
 * Returns LBM_ETIMEOUT when the timeout was recorded (the expected outcome), LBM_ECUDA if the
 * launch failed or no timeout was recorded, LBM_EINVAL for a NULL d_word. */
int lbm_selftest_wait(unsigned* d_word, void* cuda_stream);

/* The sum of lbm_reduce for callers that cannot allocate device memory.  (This entry point has no
 * counterpart in the paper; it exists for the library's users.)  Some callers may not call
 * cudaMalloc: a plugin inside a host application whose memory manager owns all device memory, code
 * that must not add an allocation (and its implicit synchronisation) while other work is in
 * flight, or a process that has spent its allocation budget.  Such a caller cannot provide the
 * workspace of lbm_create, but it may hold a population buffer in this library's layout (see
 * lbm_workspace_bytes), e.g. the current buffer of another component's handle or a checkpoint
 * already in device memory.  This call sums phi (LBM_SUM_PHI) or psi (LBM_SUM_PSI) of that buffer
 * in FP64 exactly like lbm_reduce does once a step has been taken (each cell's own slots), with its
 * partial sums in a fixed device array compiled into the library instead of a workspace.  A buffer
 * that lbm_init_fields has just filled holds, next to a wall, some values in the wall's ghost rows
 * (staged for the first pull), so its own slots give the total only after a step.
 *   d_pops: device pointer to one FP32-storage population buffer of an nx x ny grid, in the
 *           layout of lbm_workspace_bytes (read only).
 *   out:    host memory, receives the sum.
 *   cuda_stream: stream on which the work is enqueued; the call waits for it (synchronous).
 * Limit: ny <= LBM_NOALLOC_MAX_ROWS (one partial sum per row); larger grids return LBM_EINVAL
 * with a message.  nx >= 2, ny >= 2, nx * ny <= 2^30.
 * The fixed array (LBM_NOALLOC_MAX_ROWS + 1 doubles, about 64 KB) exists once per GPU that loads
 * the library and stays there until the process exits.  Its address is looked up by the first
 * call in each CUDA context (normally the primary context of the current device; a caller that
 * makes its own context current gets that context's copy), so make that first call before any
 * stream capture.
 * All calls share the array: calls that overlap on the GPU (other streams, other threads) race and
 * must be serialised by the caller.  Each call writes every entry it reads, so nothing carries over
 * from the previous call.  No device memory is allocated or freed. */
#define LBM_NOALLOC_MAX_ROWS 8192
int lbm_reduce_noalloc(const void* d_pops, int nx, int ny, int what, void* cuda_stream, double* out);

/* LBM_OK, or LBM_EUNSTABLE if the device has flagged an unstable state since lbm_init_fields.
 * Synchronous. */
int lbm_status(lbm_handle* h);

/* Checkpoint: the populations, the velocity history and the step bookkeeping, as an opaque
 * blob of lbm_state_bytes bytes in host memory.  lbm_set_state restores a blob taken from a
 * handle with identical parameters; a blob of another grid, storage mode, velocity mode or density
 * mode returns LBM_EINVAL.  Both synchronous.  n steps, a checkpoint, then n more steps give
 * bitwise the same state as 2n steps. */
int lbm_state_bytes(const lbm_handle* h, size_t* bytes);
int lbm_get_state(lbm_handle* h, void* host_blob, size_t bytes);
int lbm_set_state(lbm_handle* h, const void* host_blob, size_t bytes);

/* Number of steps taken since lbm_init_fields (or restored by lbm_set_state). */
int lbm_steps_taken(const lbm_handle* h, int64_t* steps);

/* Free the handle (not the workspace).  Waits for the handle's stream.  NULL is allowed. */
int lbm_destroy(lbm_handle* h);

/* Step kernel of a handle.  Both variants compute the same step bit for bit; they differ in how
 * the work is laid out on the GPU (FP32 storage: one cell per thread, tiles of 32 x 8 cells;
 * 16-bit storage: two horizontally adjacent cells per thread, tiles of 32 x 8 cells):
 *   LBM_KERNEL_TILE       one CTA per tile, launched as a grid of all tiles;
 *   LBM_KERNEL_PIPELINED  persistent, warp-specialised CTAs (as many as fit on all SMs, at most
 *                         one per tile): a copy warp claims tiles and stages each with TMA into
 *                         one of two buffers while the compute warps work on the other;
 *   LBM_KERNEL_AUTO       (lbm_set_kernel only) the library's choice, the faster one on GB300
 *                         at 2048 x 1024 cells: PIPELINED for 16-bit storage and for a density
 *                         ratio != 1, TILE for FP32 storage at uniform density.
 * A new handle uses the library's choice.  LBM_EINVAL if the pipelined kernel does not fit. */
#define LBM_KERNEL_AUTO 0
#define LBM_KERNEL_TILE 1
#define LBM_KERNEL_PIPELINED 2
int lbm_set_kernel(lbm_handle* h, int variant);
int lbm_get_kernel(const lbm_handle* h, int* variant);

/* Message describing the last failing call on this host thread ("" if none).  The pointer is
 * valid until the next call on the same thread. */
const char* lbm_last_error(void);

/* ---- many lattices in one launch per step --------------------------------------------------
 * Not in the paper, which treats one lattice at a time: a batch advances many independent
 * lattices (lbm_handle members, each with its own parameters, grid and workspace) by one launch
 * of one kernel per step and per group of members that share storage mode, boundary kind and
 * EOS.  Every member's result is bit for bit the one lbm_step gives it alone: a cell's update
 * depends only on its lattice's buffers, constants and step count, never on the schedule.
 * Ownership: the caller owns the batch workspace and the members; members stay valid and are
 * not destroyed while they belong to a batch (lbm_batch_set_members replaces the list).  All
 * members are created on the batch's stream.  Between batch calls a member may be used through
 * the single-lattice calls (lbm_get_moments, lbm_reduce, lbm_status, lbm_get_state, and also
 * lbm_step, lbm_init_fields, lbm_set_state): the batch reads each member's step count and
 * current buffer at the start of every lbm_batch_step.                                        */
typedef struct lbm_batch lbm_batch;

#define LBM_SCHED_MEMBER_ORDER 0     /* tiles lattice by lattice, in member order              */
#define LBM_SCHED_LARGEST_FIRST 1    /* lattice by lattice, the one with most tiles first      */
#define LBM_SCHED_EDGES_FIRST 2      /* the edge tile rows of all lattices, then the interiors */
#define LBM_SCHED_ROW_INTERLEAVED 3  /* tile row r of every lattice, then row r + 1            */
/* Within a lattice the two edge tile rows always come before the interior rows. */

/* Total tiles (ceil(nx/32) * ceil(ny/8) per lattice) of n members. */
int lbm_batch_tiles(lbm_handle* const* members, int n, int64_t* tiles);

/* Device workspace of a batch of up to max_members lattices with up to max_tiles tiles in total:
 * one descriptor per member (TMA maps, constants, buffer pointers, step count), the tile list and
 * the two tile counters of the warp-specialised kernel, each 256-byte aligned. */
int lbm_batch_workspace_bytes(int max_members, int64_t max_tiles, size_t* bytes);

/* Create an empty batch enqueuing its work on cuda_stream.  CUDA graphs (lbm_batch_set_schedule)
 * need a created stream: on the legacy default stream (NULL) graph_steps is forced to 0. */
int lbm_batch_create(int max_members, int64_t max_tiles, void* d_workspace, size_t bytes, void* cuda_stream,
                     lbm_batch** out);

/* Replace the member list (n <= max_members distinct handles, at most max_tiles tiles, each
 * lattice at most 65535 tiles along an axis; n = 0 empties the batch). */
int lbm_batch_set_members(lbm_batch* b, lbm_handle* const* members, int n);

/* Order of the tiles (LBM_SCHED_*) and the number of steps per captured CUDA graph (0: plain
 * launches).  Default: LBM_SCHED_LARGEST_FIRST, no graph. */
int lbm_batch_set_schedule(lbm_batch* b, int schedule, int graph_steps);

/* Advance every member by n steps (asynchronous, like lbm_step).  Each member's device status
 * word collects its own instability flags; read it with lbm_status(member). */
int lbm_batch_step(lbm_batch* b, int64_t n);

/* Time each schedule with 16-step graphs, and the fastest of them without a graph, over about
 * trial_steps steps each, and keep the fastest.  The trials are real steps: every member
 * advances by 4 * (16 + trial_steps rounded up to a multiple of 16) + 1 + trial_steps steps
 * (without graphs, on the legacy default stream: 4 * (1 + trial_steps)).  Synchronous. */
int lbm_batch_autotune(lbm_batch* b, int trial_steps, int* schedule, int* graph_steps);

/* Kernel of the batch's launches; both give the same results bit for bit:
 *   LBM_KERNEL_TILE       one CTA per tile of the tile list;
 *   LBM_KERNEL_PIPELINED  persistent, warp-specialised CTAs: a copy warp claims tiles from a
 *                         counter in the workspace and stages each tile's boxes and its lattice's
 *                         constants while the compute warps work on the previous tile;
 *   LBM_KERNEL_AUTO       the default: PIPELINED for every group (the faster one on GB300
 *                         with a 64-lattice mix in every storage mode).
 * PIPELINED applies only if it fits (else TILE).  lbm_batch_get_kernel reports the setting. */
int lbm_batch_set_kernel(lbm_batch* b, int variant);
int lbm_batch_get_kernel(const lbm_batch* b, int* variant);

/* Kernels this batch has launched so far (a graph replay counts its kernels). */
int lbm_batch_launches(const lbm_batch* b, int64_t* launches);

/* Free the batch (host memory only; the workspace and the members stay the caller's). */
int lbm_batch_destroy(lbm_batch* b);

/* ---- lattice server (continuous batching) --------------------------------------------------
 * Not in the paper: a job is one lattice (parameters, initial fields, step count); jobs are
 * submitted from any host thread and run by one worker thread that keeps all admitted jobs in one
 * many-lattice batch.  Each round advances every active job by one chunk of steps (cut so that no
 * job passes its step count); finished jobs leave with their final fields copied out and queued
 * jobs join at the next round.  Results are bit for bit those of the job run alone.
 * Admission: at most max_jobs active jobs with at most max_cells cells and max_tiles tiles in
 * total (a job alone may exceed max_cells), whose workspaces fit the job arena (first fit).
 * LBM_SERVE_FCFS admits in submission order (a job that does not fit blocks those behind it);
 * LBM_SERVE_SHORTEST_FIRST admits the queued job with the least work (cells x steps) first.     */
typedef struct lbm_server lbm_server;

#define LBM_SERVE_FCFS 0
#define LBM_SERVE_SHORTEST_FIRST 1

typedef struct lbm_server_config {
    int32_t policy;        /* LBM_SERVE_FCFS or LBM_SERVE_SHORTEST_FIRST                      */
    int32_t max_jobs;      /* active jobs at most (>= 1)                                      */
    int64_t max_cells;     /* active cells at most (>= 1)                                     */
    int64_t max_tiles;     /* tiles of all active jobs at most (>= 1); sizes the batch        */
    int64_t chunk_steps;   /* steps per round at most (>= 1)                                  */
    int32_t graph_steps;   /* steps per captured CUDA graph of the batch (0: plain launches) */
    int32_t schedule;      /* tile order of the batch, LBM_SCHED_*                            */
} lbm_server_config;

typedef struct lbm_job_result {
    int64_t id;
    int32_t status;        /* LBM_OK, or the code that ended the job                          */
    int32_t storage, nx, ny;
    int64_t steps;
    double t_submit, t_admit, t_done;  /* seconds on the server's steady clock                */
    char message[128];     /* error text when status != LBM_OK                                */
} lbm_job_result;

typedef struct lbm_server_stats {
    int64_t submitted, completed, queued, active;
    int64_t lattice_updates;  /* cells x steps advanced so far                                 */
    int64_t rounds;
    int64_t kernel_launches;  /* step, advance, init and moments kernels launched so far       */
    double busy_seconds;      /* worker time spent in rounds (launch to synchronise)          */
    double now;               /* the server's clock                                           */
} lbm_server_stats;

/* Device workspace of a server: the batch tables, then a job arena of job_arena_bytes. */
int lbm_server_workspace_bytes(const lbm_server_config* cfg, size_t job_arena_bytes, size_t* bytes);

/* Start a server (and its worker thread) on the current device.  The workspace (device memory,
 * 256-byte aligned) and the stream (a created stream, not NULL) are the caller's and must
 * outlive the server; everything the server launches goes to that stream. */
int lbm_server_create(const lbm_server_config* cfg, void* d_workspace, size_t bytes, void* cuda_stream,
                      lbm_server** out);

/* Queue a job.  The five initial fields (host, row-major ny x nx doubles, as lbm_init_fields) and
 * the non-NULL entries of out (host arrays receiving phi, psi, ux, uy, P at the end, as
 * lbm_get_moments) stay valid and untouched until the job's result has been polled.  Fails with
 * LBM_EINVAL for bad parameters or a job that can never fit; *id is the job's id (> 0). */
int lbm_server_submit(lbm_server* s, const lbm_params* p, const double* phi, const double* psi, const double* ux,
                      const double* uy, const double* P, int64_t steps, double* const out[5], int64_t* id);

/* Move up to max finished jobs' results into out (*n of them), waiting up to timeout_s seconds
 * for the first one (0: do not wait).  Results come in completion order. */
int lbm_server_poll(lbm_server* s, lbm_job_result* out, int max, double timeout_s, int* n);

int lbm_server_get_stats(lbm_server* s, lbm_server_stats* out);

/* Stop the worker after its current round; jobs not finished end with LBM_ESTATE (their results
 * are dropped with the server).  Frees host memory only. */
int lbm_server_destroy(lbm_server* s);

#ifdef __cplusplus
}
#endif
#endif /* GB300_LBM_H */
