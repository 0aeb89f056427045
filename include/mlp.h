/*
 * libmlp — energy and forces of an ANI-2x-shaped machine-learning potential
 * on one B300 GPU (sm_103a).
 *
 * The library evaluates the operation the paper builds its NNPOps/TorchForce
 * stack around (paper, section "PyTorch Model Support": a model takes atomic
 * positions and returns the potential energy, forces follow from the energy
 * by backpropagation or are returned explicitly; section "Optimization
 * Through NNPOps": the accelerated steps are the neighbor list and the ANI
 * atom-centered symmetry functions; section "OpenMM-ML": ANI-2x over the seven
 * elements H, C, N, O, S, F, Cl). One evaluation runs, in this library's own
 * CUDA kernels:
 *   1. staging: coordinates (FP64) -> split FP32 hi/lo, periodic wrap,
 *      species counting for the element-grouped network tiles;
 *   2. neighbor list: cell list (periodic or open systems) or all pairs
 *      within each molecule (batches of small molecules);
 *   3. atomic environment vectors (AEV): 112 radial + 896 angular terms;
 *   4. per-element networks 1008-256-192-160-1 (CELU, alpha 0.1) and their
 *      backward to dE/dG: FP32 SIMT GEMMs, or BF16 tcgen05 tensor-core GEMMs
 *      with FP32 accumulation;
 *   5. AEV backward to forces, accumulated per atom in FP64;
 *   6. per-molecule FP64 energy sums and the force output.
 *
 * Conventions
 *   Units: positions and box lengths in Angstrom, energy in the network's
 *   units (eV with trained weights), forces in energy / Angstrom.
 *   Species codes: H=0, C=1, N=2, O=3, S=4, F=5, Cl=6.
 *   Coordinates are FP64 arrays [n][3]; forces are FP32 [n][3] = -dE/dr.
 *   Boxes are orthorhombic: cell = {Lx, Ly, Lz}, or NULL for open boundary.
 *   "Host" pointers are ordinary CPU memory owned by the caller; the library
 *   copies what it needs before returning (or, for mlp_submit, before the
 *   call returns). "Device" pointers are CUDA global memory on the current
 *   device, owned by the caller, valid until the stream work completes.
 *   Streams are cudaStream_t passed as void* (NULL = the legacy stream).
 *   Handles are owned by the library and released by the matching destroy.
 *
 * Errors: every int-returning call returns MLP_OK (0) or a negative code and
 * records a message retrievable with mlp_last_error() (thread-local).
 * Invalid arguments never reach a kernel. There is no CPU fallback: without
 * a usable CUDA device every call that computes returns MLP_ECUDA.
 */
#ifndef MLP_H
#define MLP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MLP_API __attribute__((visibility("default")))
#else
#define MLP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MLP_OK = 0,
    MLP_PENDING = 1,     /* mlp_poll: the request is not finished yet            */
    MLP_EINVAL = -1,     /* bad argument (NULL, n <= 0, NaN, unknown species ...) */
    MLP_ENOMEM = -2,     /* device or host allocation failed                      */
    MLP_EAGAIN = -3,     /* server queue full or request larger than the budget   */
    MLP_ETIMEDOUT = -4,  /* mlp_wait deadline passed                              */
    MLP_ECUDA = -5,      /* CUDA runtime error (message has the CUDA error text)  */
    MLP_ENOTFOUND = -6,  /* unknown ticket                                        */
    MLP_EOVERFLOW = -7   /* neighbor capacity exceeded and could not be grown     */
};

/* Network precision. MLP_FP32: FP32 GEMMs on the CUDA cores. MLP_BF16: BF16
 * tensor-core GEMMs with FP32 accumulation; the forward (energy) GEMMs take
 * both operands as BF16 hi/lo pairs (X = X_hi + X_lo) and accumulate
 * A_hi B_hi + A_lo B_hi + A_hi B_lo, the backward (forces) single BF16
 * operands. MLP_BF16_1PASS: single BF16 operands everywhere (faster, energy
 * error ~1e-3 relative from operand rounding). AEV and forces are FP32 in
 * every mode; energy and force sums FP64. */
enum { MLP_FP32 = 0, MLP_BF16 = 1, MLP_BF16_1PASS = 2 };

#define MLP_NSPECIES 7
#define MLP_AEV_LEN 1008

typedef struct mlp_weights mlp_weights;
typedef struct mlp_system mlp_system;
typedef struct mlp_batch mlp_batch;
typedef struct mlp_server mlp_server;
typedef uint64_t mlp_ticket;

/* Host FP32 weights of the seven per-element networks, element-major:
 * W1[7][256][1008] b1[7][256] W2[7][192][256] b2[7][192] W3[7][160][192]
 * b3[7][160] W4[7][160] b4[7]; row index = output unit (y = W x + b).
 * With n_nets > 1 (ensemble, paper section "Performance of MLPs": ANI-2x is
 * an average of eight independently trained nets) every array gains a
 * leading [n_nets] axis. */
typedef struct {
    const float *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;
} mlp_weights_host;

/* Cutoffs in Angstrom. rc_rad = 5.1 and rc_ang = 3.5 are the AEV's own
 * hyper-parameters and must be given as such; skin >= 0 widens the stored
 * neighbor list (list radius rc_rad + skin) so that it can be reused across
 * calls while no atom has moved more than skin / 2. */
typedef struct {
    double rc_rad;
    double rc_ang;
    double skin;
} mlp_cutoffs;

/* ------------------------------------------------------------------ weights */

/* Uploads the weights to the current device in FP32 and BF16 with the
 * transposed copies the backward needs. n_nets in [1, 8]. With n_nets = K > 1
 * every evaluation made with these weights is the ensemble model: each atom's
 * energy is the mean of the K nets' outputs and dE/dG the mean of their
 * gradients, so energies and forces are the means over the K nets (one AEV,
 * K network passes). Returns MLP_EINVAL on NULL arrays, a non-finite W1 entry
 * or n_nets out of range, MLP_ENOMEM, MLP_ECUDA. */
/* Passage: section "OpenMM-ML" (ANI-2x: one net per element of H, C, N, O,
 * S, F, Cl) and section "Performance of MLPs" (ensemble average). */
MLP_API int mlp_weights_create(const mlp_weights_host *w, int n_nets, mlp_weights **out);
MLP_API void mlp_weights_destroy(mlp_weights *w);

/* ------------------------------------------------------------------ one system */

/* Creates a persistent system (one molecule or one periodic box) of n atoms
 * with fixed species[n]; coords[n][3] (host, may be NULL) are stored as the
 * current positions. cell = NULL gives an open boundary; otherwise every box
 * length must be >= 2 (rc_rad + skin). precision = MLP_FP32, MLP_BF16 or
 * MLP_BF16_1PASS (see the precision enum). Device buffers
 * are sized for n atoms at creation. The weights must outlive the system. */
/* Passage: section "Optimization Through NNPOps" (the neighbor list and the
 * symmetry functions are built for the system's atoms, box and cutoffs).
 * Neighbor rows hold 160 entries (256 with a skin); a host-path evaluation
 * that finds more grows them to 256 and repeats itself. */
MLP_API int mlp_create(const int8_t *species, const double *coords, int32_t n, const double *cell,
               const mlp_cutoffs *cut, const mlp_weights *w, int precision, mlp_system **out);
MLP_API void mlp_destroy(mlp_system *s);

/* One evaluation from host memory: copies coords (host [n][3]; NULL = the
 * stored positions) to the device, evaluates, and copies the energy (host
 * scalar) and forces (host [n][3], may be NULL) back. Synchronous. */
/* Passage: section "PyTorch Model Support" (positions in, potential energy
 * out, forces as the negative energy gradient). */
MLP_API int mlp_energy_forces(mlp_system *s, const double *coords, double *energy, float *forces);

/* One evaluation from device memory, asynchronous on `stream`:
 * d_coords [n][3] FP64, d_energy FP64 scalar, d_forces FP32 [n][3] (may be
 * NULL). Returns after enqueueing; the neighbor capacity check is read back
 * on the next call (or by mlp_sync), which then reports MLP_EOVERFLOW if a
 * list was truncated. */
/* Passage: section "PyTorch Model Support", as mlp_energy_forces. */
MLP_API int mlp_energy_forces_device(mlp_system *s, const double *d_coords, double *d_energy, float *d_forces,
                             void *stream);

/* ML/MM mechanical embedding (paper, section "OpenMM-ML": a mixed system
 * models a listed subset of the atoms with the MLP and everything else,
 * including the interaction between the two regions, with a conventional
 * force field that the caller supplies). s holds the n ML-region atoms
 * (created with their elements, in the order of d_index); d_index [n] int32
 * (device) gives their rows in d_coords_full [n_full][3] FP64 (device). One
 * evaluation, asynchronous on `stream`: the region's positions are gathered
 * into the system's own buffer (they become its stored positions), the
 * region is evaluated on its own (the system's cell or open boundary),
 * d_energy (FP64 scalar) receives the ML energy, and the ML forces go to rows
 * d_index of d_forces_full [n_full][3] FP32 (device; may be NULL): added to
 * what the caller placed there when accumulate != 0 (e.g. the classical
 * forces), written over those rows otherwise; other rows are not touched.
 * Returns MLP_EINVAL for NULL arguments or n_full outside [n, 2^31). An index
 * outside [0, n_full) is flagged on the device (its row is skipped) and
 * reported as MLP_EINVAL by the next call or mlp_sync; indices must be
 * distinct (a repeated row would be updated twice). */
MLP_API int mlp_energy_forces_subset_device(mlp_system *s, const double *d_coords_full, int64_t n_full,
                                            const int32_t *d_index, double *d_energy, float *d_forces_full,
                                            int accumulate, void *stream);

/* ------------------------------------------------------------------ dynamics */

/* Langevin dynamics of a system with the LF-Middle discretization (paper,
 * section "New Integrators"; the ML runs of section "Performance of MLPs",
 * Table 3, use a Langevin integrator with a 2 fs step). Velocities live at
 * half steps; one step from forces F(x_t) (eV/A), masses m (amu) of the
 * elements (H 1.008, C 12.011, N 14.007, O 15.999, S 32.06, F 18.998,
 * Cl 35.45):
 *   v <- v + dt F / m;  x <- x + dt/2 v;  v <- a v + sqrt((1 - a^2) kT / m) R;
 *   x <- x + dt/2 v;    a = exp(-friction dt)
 * in A, fs, amu, eV (F / m: 1 eV/(A amu) = 9.648533212e-3 A/fs^2; kT / m:
 * 1 eV/amu = 1 / 103.6426965 A^2/fs^2; k_B = 8.617333262e-5 eV/K). The three
 * normal deviates R of atom i at step t come from Philox4x64-10 (Salmon et
 * al., SC 2011) with counter (t, i, 0, 0) and key (seed, 0): its words w0..w3
 * give u_q = (w_q >> 11) 2^-53 and, by Box-Muller, R = sqrt(-2 ln(1 - u0))
 * (cos 2 pi u1, sin 2 pi u1) and sqrt(-2 ln(1 - u2)) cos 2 pi u3. A trajectory
 * is therefore a function of (x0, v0, seed, first step index) only. */
typedef struct mlp_langevin mlp_langevin;
typedef struct {
    double dt_fs;            /* step, > 0 */
    double friction_per_ps;  /* gamma >= 0 (0: leapfrog, no thermostat) */
    double temperature_K;    /* >= 0 */
    uint64_t seed;           /* Philox key */
    int use_graph;           /* != 0: capture one step as a CUDA graph and replay it */
} mlp_langevin_params;

/* Creates an integrator for system s (which it uses for the forces; s must
 * outlive it). MLP_EINVAL for NULL arguments or dt <= 0, friction < 0,
 * temperature < 0; MLP_ENOMEM. */
MLP_API int mlp_langevin_create(mlp_system *s, const mlp_langevin_params *p, mlp_langevin **out);
MLP_API void mlp_langevin_destroy(mlp_langevin *L);

/* Runs n_steps steps after the work queued on `stream` and waits for them
 * (graph mode replays on the integrator's own stream): d_x [n][3] and d_v
 * [n][3] FP64 (device; positions in A, velocities in A/fs at the half step
 * before), updated in place; steps are numbered step0 .. step0 + n_steps - 1
 * (the Philox counter); d_energy (device FP64 [n_steps], may be NULL)
 * receives the potential energy at the start of each step. With use_graph
 * the first run on a buffer set captures one step and every later step is a
 * graph replay (re-captured when d_x, d_v or d_energy change).
 * The system's neighbor list is rebuilt on the first step and then, with a
 * skin, whenever an atom has moved more than half the skin (device check);
 * without a skin on every step. Errors of any step (neighbor capacity,
 * network kernel) are reported at the end of the run. */
MLP_API int mlp_langevin_run(mlp_langevin *L, double *d_x, double *d_v, int64_t step0, int32_t n_steps,
                             double *d_energy, void *stream);

/* Kernel-level access for tests: the three normal deviates of atoms 0..n-1
 * at step `step` (host FP64 [n][3] out), from the device generator. */
MLP_API int mlp_debug_langevin_normals(uint64_t seed, int64_t step, int32_t n, double *normals);

/* Forward only (autograd forward): d_energy = E(d_coords). keep_aev != 0
 * keeps the AEVs on the device for a following mlp_backward_device on the
 * same coordinates; otherwise the backward recomputes them. */
/* Passage: section "PyTorch Model Support" (forces through backpropagation). */
MLP_API int mlp_forward_device(mlp_system *s, const double *d_coords, double *d_energy, int keep_aev, void *stream);

/* Backward (autograd backward): d_grad_coords[n][3] (FP32) =
 * (*d_grad_energy) * dE/dr at d_coords, with d_grad_energy an FP64 device
 * scalar (NULL = 1). Uses kept AEVs when the last forward kept them for
 * these coordinates, else recomputes them. */
MLP_API int mlp_backward_device(mlp_system *s, const double *d_coords, const double *d_grad_energy,
                        float *d_grad_coords, void *stream);

/* Waits for the system's stream work and reports a deferred error. */
MLP_API int mlp_sync(mlp_system *s);

/* ------------------------------------------------------------------ batches */

/* A batch engine for many independent open-boundary molecules of at most
 * max_atoms_per_mol atoms each (all-pairs neighbor search inside each
 * molecule), sized for max_atoms atoms and max_mols molecules in total. */
/* Passage: section "PyTorch Model Support" (the same evaluation for many
 * independent molecules at once). */
MLP_API int mlp_batch_create(const mlp_weights *w, int precision, int32_t max_atoms, int32_t max_mols,
                     int32_t max_atoms_per_mol, mlp_batch **out);
MLP_API void mlp_batch_destroy(mlp_batch *b);

/* Evaluates n_mols molecules packed back to back, all pointers device:
 * d_mol_start[n_mols + 1] (int32, d_mol_start[0] = 0, ascending), the
 * host copy of the total atom count n_atoms, d_species[n_atoms] (int8),
 * d_coords[n_atoms][3] (FP64); writes d_energy[n_mols] (FP64) and
 * d_forces[n_atoms][3] (FP32). Asynchronous on `stream`. */
MLP_API int mlp_batch_run_device(mlp_batch *b, int32_t n_mols, int32_t n_atoms, const int32_t *d_mol_start,
                         const int8_t *d_species, const double *d_coords, double *d_energy, float *d_forces,
                         void *stream);

/* Same from host memory, synchronous (pinned staging inside the batch). */
MLP_API int mlp_batch_run(mlp_batch *b, int32_t n_mols, const int32_t *mol_start, const int8_t *species,
                  const double *coords, double *energy, float *forces);

/* Returns the batch's deferred status (neighbor overflow) after its stream
 * work completed; 0 if fine. */
MLP_API int mlp_batch_sync(mlp_batch *b);

/* ------------------------------------------------------------------ serving */

typedef struct {
    int precision;              /* MLP_BF16 (default), MLP_BF16_1PASS or MLP_FP32         */
    int32_t max_batch_atoms;    /* atoms packed into one device batch (default 131072)   */
    int32_t max_batch_mols;     /* molecules per batch (default 4096)                    */
    int32_t max_atoms_per_mol;  /* largest admissible molecule (default 256)             */
    int32_t streams;            /* batches in flight on the device (default 3)           */
    int32_t queue_capacity;     /* requests outstanding (submitted, not yet collected) before MLP_EAGAIN (default 65536) */
    int64_t budget_bytes;       /* device bytes the in-flight batches may hold (40e9)    */
    /* Batching while the device is busy: with another batch in flight, a
     * free slot waits until min_batch_atoms atoms are queued or the oldest
     * queued request has waited max_wait_us, so that batches stay large
     * under load; with the device idle a batch starts at once. min_batch_atoms
     * <= 0 launches greedily. Defaults 16384 and 500. */
    int32_t min_batch_atoms;
    int32_t max_wait_us;
} mlp_server_opts;

/* Fills opts with the defaults above. */
MLP_API void mlp_server_opts_default(mlp_server_opts *opts);

/* Starts a serving loop (one host thread) that packs queued molecules into
 * batches, runs up to `streams` batches concurrently on the device, and
 * completes tickets. Device memory for all slots is reserved here, within
 * budget_bytes (MLP_ENOMEM if the slots do not fit). */
/* Passage: none in the paper, which evaluates one system per simulation
 * step; the serving loop runs the evaluation of section "PyTorch Model
 * Support" for a stream of independent requests. */
MLP_API int mlp_server_create(const mlp_weights *w, const mlp_server_opts *opts, mlp_server **out);
MLP_API void mlp_server_destroy(mlp_server *s);

/* Queues one open-boundary molecule (host species[n], coords[n][3], copied
 * before returning). Never blocks: MLP_EAGAIN when the queue is full,
 * MLP_EINVAL for n outside [1, max_atoms_per_mol] or bad input. */
/* Passage: as mlp_server_create. */
MLP_API int mlp_submit(mlp_server *s, int32_t n, const int8_t *species, const double *coords, mlp_ticket *out);

/* Non-blocking: MLP_PENDING while in flight; MLP_OK once done, writing the
 * energy and forces (host [n][3], may be NULL) and releasing the ticket. */
MLP_API int mlp_poll(mlp_server *s, mlp_ticket t, double *energy, float *forces);

/* Blocking with a deadline: MLP_ETIMEDOUT if not done within timeout_ns
 * (the ticket stays valid). */
MLP_API int mlp_wait(mlp_server *s, mlp_ticket t, int64_t timeout_ns, double *energy, float *forces);

typedef struct {
    int64_t submitted, completed, batches, atoms;
    int64_t inflight_bytes, peak_inflight_bytes;  /* device bytes held by batches in flight */
    double mean_batch_atoms;
    int64_t slot_bytes;                           /* device bytes reserved per slot        */
    int32_t slots;                                /* slots created (<= streams, by budget) */
} mlp_server_stats;

MLP_API int mlp_server_get_stats(mlp_server *s, mlp_server_stats *out);

/* Latencies (ns, submit to completion) of requests completed since the last
 * call, oldest first; copies up to cap of them into out and returns how many
 * were copied (the rest are dropped). */
MLP_API int mlp_server_latencies(mlp_server *s, int64_t *out, int cap);

/* Open-loop load generator: a native thread submits request r (molecule
 * r of the packed host arrays mol_start[n_req + 1], species, coords) at
 * arrival_ns[r] nanoseconds after the call, waits for all of them, and
 * writes energies[n_req] and forces (host [mol_start[n_req]][3], may be
 * NULL). Requests refused with MLP_EAGAIN are retried after 20 us. Returns
 * the wall time from the call to the last completion in *wall_ns. */
MLP_API int mlp_server_replay(mlp_server *s, int32_t n_req, const int64_t *arrival_ns, const int32_t *mol_start,
                      const int8_t *species, const double *coords, double *energies, float *forces,
                      int64_t *wall_ns);

/* The same with `clients` native client threads (1..64): client c submits
 * requests c, c + clients, ... at their arrival times and then collects
 * their results, as independent clients of one serving process would.
 * MLP_EINVAL for clients outside [1, 64]; a failed request or submission
 * (other than MLP_EAGAIN, which is retried) ends the replay with its code. */
MLP_API int mlp_server_replay_clients(mlp_server *s, int32_t n_req, const int64_t *arrival_ns,
                                      const int32_t *mol_start, const int8_t *species, const double *coords,
                                      double *energies, float *forces, int32_t clients, int64_t *wall_ns);

/* ------------------------------------------------------------------ allocation-free neighbor list */

/* Cell-list neighbor search for one system that allocates nothing. The paper
 * has no counterpart: this entry point exists for callers that may not call
 * cudaMalloc once they run (an engine or plugin living inside a fixed memory
 * plan or a host framework's own pool, or a time-critical loop that cannot
 * take an allocation's latency or failure). All working memory sits in a
 * file-scope __device__ array of about 2.2 MB that every GPU loading the
 * library holds until the process exits.
 *
 * d_coords [n][3] FP64 (device); cell = {Lx, Ly, Lz} (host) or NULL for an
 * open system; cutoff = list radius in A, (0, 20]; outputs (device, caller
 * owned): d_counts[n] = true neighbor count of each atom (may exceed cap),
 * d_list[n][cap] = the first min(count, cap) neighbors of each atom (all j
 * != i with |d_ij| < cutoff, minimum image when periodic). Limits: n <= 32768
 * atoms and at most 32768 cells (periodic: floor(L / cutoff) per axis);
 * larger inputs return MLP_EINVAL before any work is enqueued. Asynchronous
 * on `stream`. The first call on each device resolves the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture. Every call reuses the same array (and
 * clears its counters on `stream`), so calls that overlap on the GPU race:
 * order them on one stream or synchronize between them. */
MLP_API int mlp_neighbors_static(const double *d_coords, int32_t n, const double *cell, double cutoff,
                                 int32_t *d_counts, int32_t *d_list, int32_t cap, void *stream);

/* ------------------------------------------------------------------ memory */

/* Routes the library's device allocations through alloc_fn / free_fn (for
 * example a framework's caching allocator); NULL restores cudaMalloc. Must
 * be set before any handle is created. alloc_fn returns NULL on failure. */
MLP_API void mlp_set_allocator(void *(*alloc_fn)(size_t bytes, void *ctx), void (*free_fn)(void *ptr, void *ctx),
                       void *ctx);

/* Failure injection for tests: the after-th device allocation from now
 * (0 = the next one) fails as if the device were out of memory. */
MLP_API void mlp_debug_fail_alloc(long long after);

/* ------------------------------------------------------------------ introspection */

/* Message of the last error on this thread ("" if none). */
MLP_API const char *mlp_last_error(void);

/* Kernel launches issued by this library since load (all threads). */
MLP_API int64_t mlp_launch_count(void);

/* Per-kernel timing with CUDA events on the launching stream: enable with
 * on != 0; mlp_profile_read fills up to cap entries of name / total ms /
 * launches (names are static strings) and returns the entry count;
 * mlp_profile_reset clears the totals. Timing synchronizes each event pair,
 * so it is meant for measurement runs. */
MLP_API int mlp_profile_enable(int on);
MLP_API int mlp_profile_read(const char **names, double *total_ms, int64_t *launches, int cap);
MLP_API void mlp_profile_reset(void);

/* ------------------------------------------------------------------ kernel-level access (tests) */

/* The stored neighbor list of a system after its last evaluation: counts[n]
 * (host) and up to cap indices per atom in list[n][cap] (host); returns the
 * capacity used by the device list (call with list = NULL to query it). */
MLP_API int mlp_debug_neighbors(mlp_system *s, int32_t *counts, int32_t *list, int32_t cap);

/* AEVs of the last evaluation in atom order, host FP32 G[n][1008]: the value
 * the network consumes (FP32 path: the FP32 row; MLP_BF16: G_hi + G_lo;
 * MLP_BF16_1PASS: G_hi). */
MLP_API int mlp_debug_aev(mlp_system *s, float *G);

/* The BF16 paths' stored AEV rows of the last evaluation in atom order, each
 * BF16 value widened to FP32: G_hi[n][1008] and (MLP_BF16, may be NULL)
 * G_lo[n][1008], the BF16 rounding of G - G_hi (zero for MLP_BF16_1PASS).
 * MLP_EINVAL on an FP32-path system. */
MLP_API int mlp_debug_aev_split(mlp_system *s, float *G_hi, float *G_lo);

/* The force kernel alone (AEV backward, section "PyTorch Model Support"):
 * forces[n][3] (host FP64, the kernel's FP64 sums, negated) for the caller's
 * dEdG[n][1008] (host FP32, atom order), on the positions and neighbor list
 * of the system's last evaluation, with the arithmetic of the system's
 * precision (FP32 path: dE/dG read as FP32, library-accurate functions; BF16
 * paths: dE/dG rounded to BF16 to nearest even, the fast hardware
 * approximations). Overwrites the system's stored dE/dG and force sums; the
 * next evaluation rebuilds its neighbor list. */
MLP_API int mlp_debug_forces(mlp_system *s, const float *dEdG, double *forces);

/* Per-atom energies e[n] (host FP32) and dE/dG[n][1008] (host FP32, may be
 * NULL) of the last evaluation that ran the network backward. */
MLP_API int mlp_debug_atom_energies(mlp_system *s, float *e, float *dEdG);

/* Runs only the network (forward and backward) on caller-provided AEV rows:
 * host G[n][1008] FP32 and species[n]; writes e[n] and dEdG[n][1008] (host).
 * precision selects the FP32 SIMT or the BF16 tensor-core network. */
MLP_API int mlp_debug_network(const mlp_weights *w, int precision, int32_t n, const int8_t *species, const float *G,
                      float *e, float *dEdG);

/* Failure detection without a fault: one thread of a one-block kernel runs the
 * tensor-core kernels' bounded wait on a barrier phase that nothing completes.
 * The wait gives up after its limit (2 s), records the waiting warp and
 * barrier, and the kernel returns; *timed_out = 1 and *code = that record
 * (bit 30 set, warp in bits 20..25, barrier address below). The context
 * stays usable. MLP_ECUDA if the launch fails. */
MLP_API int mlp_debug_wait_timeout(int32_t *timed_out, int32_t *code);

#ifdef __cplusplus
}
#endif
#endif /* MLP_H */
