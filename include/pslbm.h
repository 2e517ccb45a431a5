/*
 * pslbm.h -- C ABI of the GB300 (sm_103a) library for the pore-scale
 * two-phase multi-mixture reactive lattice Boltzmann method of
 * Chen, Kang, Tang, Robinson, He, Tao (arXiv 1410.3464).
 *
 * One time step (pslbm_step) advances, on the GPU, for every lattice node:
 *   - the pseudo-potentials psi_1 (C-S EOS, Eqs. 12-13) and phi_1, phi_2
 *     (Eq. 15), the Shan-Chen cohesion, inter-component and adhesion forces
 *     (Eqs. 11, 14, 16) and the velocities of Eqs. 17-19;
 *   - the D2Q9 BGK collide-stream of the liquid and gas components with the
 *     reaction source omega_a S_sigma (Eqs. 6-8, 27) and halfway bounce-back;
 *   - liquid/gas marking against half the maximum liquid-component density
 *     (Section 4.5) with the concentration amendment at changed nodes;
 *   - the D2Q5 collide-stream of every transported solute in the liquid phase
 *     with homogeneous sources (Eqs. 20-24, 26, 28), no-flux liquid-gas links
 *     and reactive liquid-solid links (Eqs. 29-31);
 *   - the volume-of-pixel update of the solid volumes (Eqs. 32-35) and the
 *     status changes solid<->liquid with their amendment (Section 4.7, Steps 4-5).
 *
 * Conventions
 *   - Every call returns a pslbm_status; PSLBM_OK is 0, errors are negative.
 *   - Host arrays are row-major [ny][nx] (index y*nx + x), borrowed for the
 *     duration of the call and copied; outputs go to caller-owned host buffers.
 *   - Errors are sticky per handle: after a device error every call on the
 *     handle returns it; pslbm_last_error() gives a message.  pslbm_destroy()
 *     is always safe.
 *   - Work is queued on the library stream (pslbm_get_stream / pslbm_set_stream)
 *     and is asynchronous; pslbm_read_fields and pslbm_sync synchronise it.
 *   - Calls on one handle are not thread-safe; distinct handles may be used
 *     from distinct threads only if they are not in the same batch.
 */
#ifndef PSLBM_H
#define PSLBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pslbm_s* pslbm_t;          /* one simulation, owned by the library */
typedef struct pslbm_batch_s* pslbm_batch_t; /* a group of simulations stepped together */

typedef enum {
    PSLBM_OK = 0,
    PSLBM_ERR_PARAM = -1,       /* invalid argument or parameter set */
    PSLBM_ERR_OOM = -2,         /* device or host allocation failed (nothing leaked) */
    PSLBM_ERR_CUDA = -3,        /* CUDA runtime error (message in pslbm_last_error) */
    PSLBM_ERR_NONFINITE = -4,   /* a density became NaN/Inf on the device */
    PSLBM_ERR_EOS_DOMAIN = -5,  /* Eq. 13 square-root argument negative (rho_1 out of the EOS domain) */
    PSLBM_ERR_TIMEOUT = -6,     /* a bounded device-side wait gave up */
    PSLBM_ERR_STATE = -7,       /* call not valid in the handle's current state */
    PSLBM_ERR_NODEVICE = -8     /* no CUDA device, or not an sm_103 device */
} pslbm_status;

typedef enum {
    PSLBM_FP64 = 0,              /* populations stored and computed in FP64 */
    PSLBM_FP32 = 1,              /* FP32 compute, populations stored as f - w_a rho_ref(phase) (shifted) */
    PSLBM_FP32_SOLUTE_F16 = 2,   /* as FP32, solute populations stored in IEEE half */
    PSLBM_FP32_SOLUTE_BF16 = 3   /* as FP32, solute populations stored in bfloat16 */
} pslbm_precision;

/* Node types (Fig. 2: liquid, gas, solid D(s), solid F(s); plus inert walls and
 * reservoir nodes that push a fixed equilibrium state into their neighbours). */
enum {
    PSLBM_LIQUID = 0, PSLBM_GAS = 1, PSLBM_SOLID_D = 2, PSLBM_SOLID_F = 3,
    PSLBM_WALL = 4, PSLBM_INLET = 5, PSLBM_OUTLET = 6
};

#define PSLBM_MAX_SPECIES 4
#define PSLBM_IDX_ABSENT (-1)
#define PSLBM_IDX_DERIVED (-2)

/* Parameter block.  struct_size must be sizeof(pslbm_params). */
typedef struct {
    uint32_t struct_size;
    int32_t nx, ny;                /* lattice size, nx, ny >= 1, nx*ny <= 100,000,000 */
    int32_t periodic_x, periodic_y;/* 1: periodic axis; 0: outside the edge acts as a wall */
    int32_t precision;             /* pslbm_precision */
    /* fluid: Eqs. 6-19 */
    double tau[2];                 /* BGK relaxation times (> 0.5), liquid and gas component */
    double G11, G12, G21;          /* Eq. 11 cohesion (G22 = 0), Eq. 14 cross interactions */
    double a0, rho10, rho20;       /* Eq. 15 constants */
    double w_adh[2];               /* Eq. 16 fluid-solid interaction strengths; with 0 a wall
                                      holds a 90-degree contact angle (solid neighbours enter
                                      the Eq. 11 and 14 sums as their mirror images across the
                                      wall), below 0 it wets */
    double eos_a, eos_b, eos_R, eos_T; /* Eq. 12 Carnahan-Starling constants and temperature */
    double body_force[2];          /* optional uniform acceleration (x, y) */
    double rho_ref[2];             /* reference densities of the liquid phase: FP32 population
                                      shift of liquid-marked nodes and the fill density of a
                                      refilled node with no fluid neighbour */
    /* solutes: Eqs. 20-24 */
    int32_t n_species;             /* transported species, 0..PSLBM_MAX_SPECIES */
    int32_t idx_A, idx_B, idx_E, idx_F; /* species index of A, B, E, F; -1 absent; A may be -2 (derived) */
    double J0[PSLBM_MAX_SPECIES];  /* rest fractions (Eq. 22), 0 <= J0 < 1 */
    double tau_g[PSLBM_MAX_SPECIES];  /* relaxation times (> 0.5) */
    double conc_ref[PSLBM_MAX_SPECIES]; /* FP32/16-bit solute population shift */
    /* reactions: Eqs. 1-5, 27-31 */
    double k1, inv_Keq, k3;        /* homogeneous R1 = k1 (C_A - inv_Keq C_B sqrt(C_C)), R3 = k3 C_B C_E */
    double k2, k4, C_F_sat;        /* heterogeneous R2 = k2 C_B at D(s), R4 = k4 (C_F - C_F_sat) at D(s)/F(s) */
    double gas_yield;              /* Eq. 27: S_2 = -S_1 = gas_yield * R1 (0.5 M_C) */
    double inv_M_C;                /* C_C = rho_2 * inv_M_C */
    double c_total_per_rho1;       /* derived A: C_A = max(0, c_total_per_rho1 rho_1 - sum_k C_k) */
    /* volume of pixel: Eqs. 32-35 */
    double Vbar_D, Vbar_F;         /* molar volumes of D(s), F(s) */
    double V_split;                /* overflow threshold of V_D + V_F (> 1) */
    uint64_t seed;                 /* seed of the overflow-neighbour choice (SplitMix64) */
    /* reservoir nodes */
    double rho_in_liq[2], rho_in_gas[2]; /* inlet densities during liquid / gas slugs */
    double rho_out[2];             /* outlet densities while the node upstream (x - 1) is liquid */
    double rho_out_gas[2];         /* outlet densities while the node upstream is gas */
    int32_t inlet_period_liq, inlet_period_gas; /* slug lengths in steps (gas 0: always liquid) */
    int32_t inlet_ramp;            /* steps of linear blend between the liquid and gas inlet
                                      states at the end of each slug (0: sharp switch) */
    double conc_in[PSLBM_MAX_SPECIES];  /* inlet concentrations */
    double r1_surface_factor;      /* Section 2: R1 runs this many times faster at the surface of
                                      D(s) -- at liquid nodes sharing an axis link with a D(s)
                                      node -- than in the bulk (0 is read as 1) */
    double rho_ref_gas[2];         /* reference densities of the gas phase: FP32 population
                                      shift of gas-marked nodes (each node's populations are
                                      stored relative to its own phase, so that both phases
                                      keep their FP32 digits at a large density ratio) */
    int32_t inlet_axis, outlet_axis; /* 0: inlet nodes feed x + 1 and outlet nodes drain x - 1;
                                      1: they feed y + 1 / drain y - 1 (a free top outlet) */
    double conc_scale[PSLBM_MAX_SPECIES]; /* 16-bit solute storage only: species k's (shifted)
                                      populations are stored multiplied by conc_scale[k], rounded
                                      to the nearest power of two (0 is read as 1), so that a
                                      trace species far below 1 keeps FP16's digits instead of
                                      falling below its range; scaling by a power of two is
                                      exact, so only the stored rounding changes.  Ignored for
                                      FP64 and FP32 storage.  Must be >= 0 and finite. */
} pslbm_params;

/* Field selectors for pslbm_read_fields; each selected field has its own
 * caller-owned host buffer in `out`, in the order of the bits below.  Doubles
 * unless noted; fields are 0 where they are not defined. */
enum {
    PSLBM_F_RHO1 = 1u << 0,      /* [ny*nx] liquid-component density (fluid nodes) */
    PSLBM_F_RHO2 = 1u << 1,      /* [ny*nx] gas-component density (fluid nodes) */
    PSLBM_F_UX = 1u << 2,        /* [ny*nx] physical velocity u_r of Eq. 19, x (fluid nodes) */
    PSLBM_F_UY = 1u << 3,        /* [ny*nx] u_r, y */
    PSLBM_F_CONC = 1u << 4,      /* [n_species*ny*nx] concentrations (liquid nodes) */
    PSLBM_F_TYPE = 1u << 5,      /* [ny*nx] uint8 node types */
    PSLBM_F_VOL = 1u << 6,       /* [2*ny*nx] V_D then V_F */
    PSLBM_F_BUDGET = 1u << 7     /* [6 + n_species]: max rho1, sum rho1, sum rho2 (fluid),
                                    sum C_k (liquid), sum V_D, sum V_F, step count (as double) */
};

/* Library stream: all device work of the library is ordered on it.  The
 * getter returns a cudaStream_t as void*.  set_stream(NULL) restores the
 * library's own stream; the caller keeps ownership of a stream it passes. */
void* pslbm_get_stream(void);
pslbm_status pslbm_set_stream(void* cuda_stream);

/* Create a simulation.
 *   mask      [ny*nx] node types (required).
 *   rho1,rho2 [ny*nx] initial densities at fluid nodes (required); populations
 *             start at the rest equilibrium of Eq. 8.
 *   conc      [n_species*ny*nx] initial concentrations at liquid nodes, or NULL (0);
 *             solute populations start at J_a C (Eq. 21 at rest).
 *   vol       [2*ny*nx] initial V_D, V_F, or NULL (1 at SOLID_D / SOLID_F nodes).
 *   p         parameters (validated: PSLBM_ERR_PARAM on invalid values, incl.
 *             tau <= 0.5, k >= (1 - J0)/2 for a reactive species, bad indices).
 * On success *out holds a new handle; on failure *out is NULL and nothing leaks.
 * The initial liquid threshold is half the maximum initial rho1 over fluid nodes.
 * The handle's device state is one allocation (pslbm_device_bytes; the tile
 * lists of the step kernels are allocated on demand); the inputs are copied
 * with cudaMemcpyAsync on the library stream (page-locked host buffers copy
 * fastest) and the call synchronises once before it returns, after which the
 * caller may reuse them. */
pslbm_status pslbm_create(const uint8_t* mask, const double* rho1, const double* rho2,
                          const double* conc, const double* vol,
                          const pslbm_params* p, pslbm_t* out);

/* Advance n >= 0 time steps (asynchronous; replays a captured CUDA graph). */
pslbm_status pslbm_step(pslbm_t h, int64_t n);

/* Wait for queued work and report any device-side status (non-finite
 * density, EOS domain) as an error. */
pslbm_status pslbm_sync(pslbm_t h);

/* Copy the selected fields (bit mask of PSLBM_F_*) to host buffers out[i]
 * (one per selected field, in bit order).  Synchronises the stream. */
pslbm_status pslbm_read_fields(pslbm_t h, uint32_t fields, void* const* out);

/* Run n >= 1 steps without graph capture, timing each kernel with CUDA
 * events on the library stream, and synchronise.  kernel_ms[3] receives the
 * mean duration per step (ms) of the bulk kernel (Eqs. 6-31 fused), the VOP
 * kernel (Eqs. 32-35) and the amendment kernel (Section 4.5); total_ms the
 * mean time per step from the first to the last event.  Same results as
 * pslbm_step. */
pslbm_status pslbm_profile_step(pslbm_t h, int64_t n, double* kernel_ms, double* total_ms);

/* Freeze the simulation once it has taken `limit` steps (limit < 0: no limit).
 * Steps requested beyond the limit leave the state unchanged, so simulations
 * with different step budgets can share one batch.  Synchronises. */
pslbm_status pslbm_set_step_limit(pslbm_t h, int64_t limit);

/* Device bytes pslbm_create would allocate for this parameter set (excluding
 * the read-back scratch of pslbm_read_fields). */
pslbm_status pslbm_estimate_device_bytes(const pslbm_params* p, uint64_t* bytes);

/* Tile shape of the step kernels, which also sets the nodes per thread of a
 * 256-thread block: 16x16 or 32x8 (one node per thread), 16x32 or 32x16 (two
 * nodes per thread: thread (tx, ty) computes rows ty and ty + 256 / tile_x).
 * (0, 0), the default, leaves the shape to timing: the next step call long
 * enough to try every open variant (tile shape x staging, 4 steps each, in
 * two passes, the second in reverse order; the steps advance the simulation
 * like any others) times them and keeps the fastest by its better pass;
 * the results do not depend on the variant.  tuned reports whether the variant
 * has been chosen (by timing, or because only one was left open).
 * PSLBM_ERR_PARAM for another shape, or for a two-node shape while staging 1
 * is fixed (the handle is left as it was). */
pslbm_status pslbm_set_tile_shape(pslbm_t h, int32_t tile_x, int32_t tile_y);
pslbm_status pslbm_get_tile_shape(pslbm_t h, int32_t* tile_x, int32_t* tile_y, int32_t* tuned);

/* Staging of the bulk kernel's populations: 0 plain per-thread loads; 1 TMA
 * copies of each tile's D2Q9 and D2Q5 population boxes into shared memory two
 * tiles ahead (two stages, two blocks per SM; one-node tile shapes only); 2
 * TMA copies of the D2Q9 box only, one tile ahead, re-read from shared memory
 * where used, with the solute populations loaded directly (two stages; three
 * blocks per SM with one node per thread, two with two, whose box has no x
 * halo).  1 and 2 are available for the FP32-population precisions
 * when a row of the lattice is a multiple of 16 bytes (nx a multiple of 4, and
 * of 8 with 16-bit solutes).  -1 (the default) leaves the choice to timing.
 * PSLBM_ERR_PARAM for 1 or 2 where they are not available, and for 1 while a
 * two-node tile shape is fixed.  The results are bit-identical either way.  get reports the
 * staging in use and whether staging is available for the handle.  A staged
 * kernel whose copy does not arrive within about a second stops and sets
 * PSLBM_ERR_TIMEOUT (sticky), reported by the next sync or read. */
pslbm_status pslbm_set_staging(pslbm_t h, int32_t mode);
pslbm_status pslbm_get_staging(pslbm_t h, int32_t* staged, int32_t* available);

/* Per-step monitor: the number of steps taken, the maximum liquid-component
 * density over fluid nodes found by the last step (the quantity whose half is
 * the next liquid threshold, Section 4.5; the initial maximum before the first
 * step) and the device status bits (1 non-finite density, 2 EOS domain,
 * 4 event-list overflow, 8 staged-copy timeout).  Reads 72 bytes from the
 * device and synchronises the library stream; no kernel runs.  Returns the
 * matching error status when a bit is set (sticky, as for pslbm_sync).  Any
 * output pointer may be NULL. */
pslbm_status pslbm_monitor(pslbm_t h, int64_t* steps, double* max_rho1, uint32_t* status);

/* Number of steps taken and lattice size. */
pslbm_status pslbm_info(pslbm_t h, int64_t* steps, int32_t* nx, int32_t* ny, int32_t* n_species);

/* Device bytes held by the handle. */
pslbm_status pslbm_device_bytes(pslbm_t h, uint64_t* bytes);

/* Release all resources of the handle (safe on NULL and on failed handles). */
pslbm_status pslbm_destroy(pslbm_t h);

/* Last error message of the handle (or of the library when h is NULL). */
const char* pslbm_last_error(pslbm_t h);

/* Budget of the current state written to DEVICE memory without allocating
 * anything.  The paper has no counterpart: this entry point exists for callers
 * that must not allocate device memory at the moment they want the budget --
 * hosts that give the library a fixed memory pool and forbid any later
 * allocation, and real-time loops where an allocation (which can synchronise
 * the device or wait on a driver lock) could stall.
 *   out  caller-owned device buffer of 6 + n_species doubles; receives the
 *        PSLBM_F_BUDGET layout (max rho1, sum rho1, sum rho2, sum C_k, sum V_D,
 *        sum V_F, step count), bit for bit the numbers pslbm_read_fields gives
 *        (same reduction grid, same order of additions).
 * Asynchronous on the library stream.  The per-block partial sums live in one
 * file-scope device array of 512 x 9 doubles (36 KiB), held by every GPU that
 * loads the library until the process exits; each of the 512 rows covers a
 * contiguous 1/512 of the lattice, so every lattice the library accepts fits
 * (up to 100,000,000 nodes) and no size is rejected.  Every call overwrites all
 * 512 rows before it reads them, so nothing has to be cleared between calls,
 * but all calls share the array: calls that overlap on the GPU (other streams,
 * other threads) race.  The first call on each device looks up the array's
 * device address (with that device current); make that first call before any
 * stream capture.  Returns the handle's sticky error, if any, without
 * launching.  Calls no cudaMalloc, cudaFree or allocating library routine. */
pslbm_status pslbm_budget_device_noalloc(pslbm_t h, double* out);

/* ---------------------------------------------------------------- batching
 * A batch steps several simulations (same precision and species count) in
 * one launch per kernel over a packed list of tiles of all members.  The
 * members stay valid handles; they must not be stepped on their own while
 * the batch exists.  tile_x, tile_y choose the tile shape (16x16, 32x8,
 * 16x32 or 32x16, as for pslbm_set_tile_shape; 0, 0: time every open variant
 * on the first steps and keep the fastest). */
pslbm_status pslbm_batch_create(int32_t n, const pslbm_t* members, int32_t tile_x, int32_t tile_y,
                                pslbm_batch_t* out);
pslbm_status pslbm_batch_step(pslbm_batch_t b, int64_t n);
pslbm_status pslbm_batch_sync(pslbm_batch_t b);
pslbm_status pslbm_batch_get_tile_shape(pslbm_batch_t b, int32_t* tile_x, int32_t* tile_y, int32_t* tuned);
/* Staging for the batch as for a single handle; available only when every
 * member has it. */
pslbm_status pslbm_batch_set_staging(pslbm_batch_t b, int32_t mode);
pslbm_status pslbm_batch_get_staging(pslbm_batch_t b, int32_t* staged, int32_t* available);
/* As pslbm_profile_step for a batch: n >= 1 steps without graph capture, each
 * kernel timed with CUDA events on the library stream; kernel_ms[3] receives
 * the mean ms per step of the bulk, VOP and amendment kernels over all
 * members, total_ms (nullable) the mean ms per step.  Synchronises. */
pslbm_status pslbm_batch_profile_step(pslbm_batch_t b, int64_t n, double* kernel_ms, double* total_ms);
/* Per-step monitor of a batch: the smallest step count over the members and
 * the OR of their device status bits (as in pslbm_monitor), gathered on the
 * device and read in one copy (16 bytes per member).  Synchronises.  The
 * status bits are reported, not raised: a member's error is returned by
 * pslbm_batch_sync or by the member's own calls once the batch is gone. */
pslbm_status pslbm_batch_monitor(pslbm_batch_t b, int64_t* min_steps, uint32_t* status);
pslbm_status pslbm_batch_destroy(pslbm_batch_t b);

/* ---------------------------------------------------------------- serving
 * Continuous batching of simulation requests.  Requests queue on the host;
 * each pslbm_server_advance() admits queued requests in arrival order while
 * the device-memory estimate of the resident simulations stays within
 * hbm_budget_bytes (and their count within max_active), re-packs the resident
 * simulations into batches when the set changed (one per species count; the
 * first batch of a species count chooses the kernel variant by timing when a
 * chunk is long enough, and the batches re-packed after it take that variant),
 * advances them by chunk_steps
 * steps (a simulation is frozen at its step budget), and retires requests that
 * reached their step budget or whose total solid volume changed by at least
 * their stop fraction (checked after each chunk).  Retired requests keep their
 * final budget (and their fields if asked) on the host until released. */
typedef struct pslbm_server_s* pslbm_server_t;
typedef struct {
    uint32_t struct_size;          /* sizeof(pslbm_server_config) */
    int32_t precision;             /* pslbm_precision of every resident simulation */
    uint64_t hbm_budget_bytes;     /* admission budget of device memory */
    int32_t chunk_steps;           /* steps per scheduling chunk (>= 1) */
    int32_t max_active;            /* resident simulation cap (>= 1) */
} pslbm_server_config;
enum { PSLBM_REQ_QUEUED = 0, PSLBM_REQ_ACTIVE = 1, PSLBM_REQ_DONE = 2, PSLBM_REQ_FAILED = 3 };

pslbm_status pslbm_server_create(const pslbm_server_config* config, pslbm_server_t* out);
/* Queue a request (inputs as in pslbm_create, copied; the server's precision
 * replaces p->precision).  step_budget >= 1; stop_dv_frac > 0 also retires the
 * request once |sum V - sum V(0)| >= stop_dv_frac * sum V(0); keep_fields != 0
 * keeps rho1, rho2, ux, uy, conc, type and vol of the final state for fetch. */
pslbm_status pslbm_server_submit(pslbm_server_t s, const uint8_t* mask, const double* rho1, const double* rho2,
                                 const double* conc, const double* vol, const pslbm_params* p,
                                 int64_t step_budget, double stop_dv_frac, int32_t keep_fields, uint64_t* req_id);
/* Run one scheduling chunk; reports resident, queued and just-retired counts.  Synchronises. */
pslbm_status pslbm_server_advance(pslbm_server_t s, int32_t* n_active, int32_t* n_queued, int32_t* n_done);
/* State (PSLBM_REQ_*), steps taken, and for a finished request its final
 * budget (6 + n_species doubles, layout of PSLBM_F_BUDGET) into budget_out (nullable). */
pslbm_status pslbm_server_poll(pslbm_server_t s, uint64_t req_id, int32_t* state, int64_t* steps_done,
                               double* budget_out);
/* Kept fields of a finished request (bits PSLBM_F_RHO1 .. PSLBM_F_VOL, buffers in bit order). */
pslbm_status pslbm_server_fetch(pslbm_server_t s, uint64_t req_id, uint32_t fields, void* const* out);
pslbm_status pslbm_server_release(pslbm_server_t s, uint64_t req_id);
const char* pslbm_server_last_error(pslbm_server_t s);
pslbm_status pslbm_server_destroy(pslbm_server_t s);

#ifdef __cplusplus
}
#endif
#endif /* PSLBM_H */
