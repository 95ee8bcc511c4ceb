/* wcsim: wavelet-compressed patch time stepping for LBM / FV schemes on one
 * GB300 (sm_103a).
 *
 * The method (Flint & Helluy, "Reducing the memory usage of Lattice-Boltzmann
 * schemes with a DWT-based compression"):
 *   - the domain is split into patches (Sec. 3.1.1); with the folded BL5/3
 *     wavelet a patch of P cells holds P+1 nodes and shares its bordering
 *     nodes with its neighbours so that mass is conserved exactly;
 *   - every patch stays in device memory only as thresholded wavelet
 *     coefficients (Sec. 2: DWT of Sec. 2.1.2, hard threshold of Sec. 2.2,
 *     lossless stage of Sec. 2.3);
 *   - every time step decodes a patch, applies one scheme step (Sec. 1, eq.
 *     vf_scheme, or a D2Q9 BGK collide-stream) and re-encodes it.  The paper
 *     decodes the whole grid each step and names per-patch decoding as future
 *     work (Sec. 3.2.4, last paragraph); that is what this library does, one
 *     fused kernel launch per time step.
 *
 * Conventions for every entry point:
 *   - every call returns a wcs_status; nothing throws across this boundary;
 *   - the caller owns every buffer it passes (host or device, as stated); the
 *     library owns all device state of a simulation and frees it in
 *     wcs_destroy;
 *   - work is enqueued on the stream given at creation (NULL = legacy default
 *     stream); calls that return data to the host synchronise that stream;
 *   - errors detected on the device (arena overflow, NaN) are sticky: they are
 *     reported by the next synchronising call (wcs_sync, wcs_stats,
 *     wcs_export_field, wcs_step with sync) and the state is left at the last
 *     completed step;
 *   - a simulation is not thread-safe: one host thread at a time.
 */
#ifndef WCSIM_H
#define WCSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wcs_sim wcs_sim;

typedef enum {
  WCS_OK = 0,
  WCS_E_ARG = 1,          /* invalid argument or combination */
  WCS_E_OOM = 2,          /* device allocation failed */
  WCS_E_ARENA_FULL = 3,   /* compressed state outgrew its arena */
  WCS_E_NAN = 4,          /* a NaN/Inf coefficient was produced */
  WCS_E_TIMEOUT = 5,      /* a bounded device wait gave up */
  WCS_E_CUDA = 6,         /* a CUDA runtime call failed */
  WCS_E_UNSUPPORTED = 7   /* no compiled kernel for this configuration */
} wcs_status;

/* Schemes.  D2Q9: 9 populations, lattice units, periodic axes only.
 * D3Q19: 19 populations on a 3-D grid (dims = 3), lattice units, periodic
 * axes only; compiled for BL5/3, FP32 compute, F32 or BF16 details, P = 32
 * or 16, L = 3.  EULER2D: (rho, rho u, rho v, E), perfect gas, Rusanov flux
 * in the form of the paper's eq. vf_scheme, periodic or outflow axes.
 * TRANSPORT: one field W, the paper's linear transport (Sec. 3.1.2) with the
 * upwind flux of eq. upwind_trans, velocity opts.velocity; compiled for
 * BL5/3, FP32 compute with F32 details, P = 64, L = 1..5, and FP64 P = 32
 * L = 3.  SWE: (h, h u, h v), shallow water with the Godunov flux of the
 * exact Riemann solver (Sec. 3.2.4), gravity opts.gravity; BL5/3, FP32/F32
 * P = 64 L = 4 and FP64 P = 32 L = 3.  The FV schemes (EULER2D, TRANSPORT,
 * SWE) take periodic or outflow (zero-gradient) axes. */
typedef enum { WCS_D2Q9 = 0, WCS_D3Q19 = 1, WCS_EULER2D = 2, WCS_TRANSPORT = 3, WCS_SWE = 4 } wcs_scheme;

/* Wavelets: folded BL5/3 on P+1 nodes (Sec. 2.1.2), Haar on P cells, or
 * CDF 9/7 on P+1 nodes (the second-order alternative Sec. 2.1.2 names;
 * lifting factorisation folded like BL5/3: the end samples are kept, so
 * shared edges decode alike in both patches; constants pass through; it
 * keeps no trapezoid mass, so field_sum is an estimate); CDF 9/7 is
 * compiled for TRANSPORT, FP32/F32, P = 64, L = 4. */
typedef enum { WCS_BL53 = 0, WCS_HAAR = 1, WCS_CDF97 = 2 } wcs_wavelet;

/* Threshold rules of Sec. 2.2 (accumulation / capped under the reading that
 * the finest band gets eps and coarser bands smaller thresholds). */
typedef enum { WCS_RULE_CONST = 0, WCS_RULE_ACCUM = 1, WCS_RULE_CAPPED = 2 } wcs_rule;

/* Storage of the surviving detail coefficients. */
typedef enum { WCS_STORE_F64 = 0, WCS_STORE_F32 = 1, WCS_STORE_BF16 = 2, WCS_STORE_I8 = 3 } wcs_store;

/* Arithmetic precision of the whole step (FP64 computes stores F64). */
typedef enum { WCS_FP64 = 0, WCS_FP32 = 1 } wcs_prec;

typedef struct {
  int dims;               /* 2, or 3 for D3Q19 */
  int64_t n[3];           /* cells per axis (multiple of the patch size) */
  uint32_t periodic_mask; /* bit a set: axis a periodic, else outflow */
} wcs_grid;

typedef struct {
  int wavelet;            /* wcs_wavelet */
  int rule;               /* wcs_rule */
  int detail_store;       /* wcs_store */
  int compute;            /* wcs_prec */
  double tau;             /* D2Q9 relaxation time (omega = 1/tau) */
  double cfl;             /* FV schemes: > 0: dt = cfl h / v_max, v_max the
                             largest signal speed of the current state
                             (EULER2D: max(|u|+c, |v|+c); SWE: the same with
                             c = sqrt(g h)) or max(|alpha|, |beta|)
                             (TRANSPORT); < 0: fixed step dt/h = -cfl */
  double gamma;           /* EULER2D ratio of specific heats */
  double arena_factor;    /* > 0: fixed arena capacity per buffer, as a
                             fraction of the uncompressed state size in the
                             compute type; an overflow is reported as
                             WCS_E_ARENA_FULL.  0: automatic: after every
                             encode of a whole state the capacity is set to
                             1.5 x the live record bytes (+ 512 B per
                             patch), synchronising calls keep it between
                             1.25 x and 2 x the live bytes, and a step whose
                             records overflowed is re-run with twice the
                             capacity (not with a learned threshold, nor
                             inside a batch) */
  void* cuda_stream;      /* cudaStream_t, NULL = default stream */
  double velocity[2];     /* TRANSPORT: (alpha, beta) */
  double gravity;         /* SWE: g (0 = 9.81) */
  double length;          /* FV schemes: side of the square domain, so that
                             h = length / cells and time = sum of dt (0 = 1) */
  int coarse_hilo;        /* 1: hi + lo coarse storage (Sec. 2.1.2, eq.
                             conservation; FP32 compute on BL5/3, 2-D and
                             D3Q19): every
                             encode also forms the coarse block in FP64 from
                             the same FP32 nodes and keeps, beside each FP32
                             coarse sample hi of the record, the FP32 part
                             lo = fl32(c64 - hi) it lacks (wcs_coarse_lo), so
                             that field_sum + field_sum_lo is the FP64 mass of
                             the nodes before the encode to about 1e-14
                             relative; the lo parts count as compressed
                             bytes.  WCS_E_UNSUPPORTED where no kernel keeps
                             them.  0: off */
} wcs_opts;

/* Per-step diagnostics, all reductions in FP64 in a fixed order. */
typedef struct {
  int64_t step;              /* completed time steps */
  double time;               /* physical time (EULER2D) or steps (D2Q9) */
  double field_sum[19];      /* per field: trapezoid-weighted sum computed
                                from the coarse coefficients (details carry
                                no mass, eq. conservation) */
  double mass;               /* D2Q9: sum of populations; EULER2D: rho;
                                TRANSPORT: W; SWE: h */
  double momentum[3];        /* D2Q9: sum c_i f_i; EULER2D: rho u, rho v;
                                SWE: h u, h v */
  double energy;             /* EULER2D: E */
  double smax;               /* EULER2D, SWE: largest signal speed of the
                                state (0 with a fixed step, cfl < 0, on
                                BL5/3, where no step needs it) */
  int64_t live_bytes;        /* bytes of the records of the current state */
  int64_t resident_bytes;    /* every device byte the simulation holds */
  int64_t uncompressed_bytes;/* one uncompressed copy of the state */
  uint32_t status;           /* sticky device status bits */
  int64_t arena_capacity;    /* bytes of each of the two record arenas */
  int64_t arena_reruns;      /* steps re-run after an arena overflow (auto
                                arenas), since creation */
  double field_sum_lo[19];   /* coarse_hilo: per field the lo parts' share,
                                2^(dims L) times their trapezoid sum (0 when
                                off); field_sum + field_sum_lo is the FP64
                                coarse-domain mass */
} wcs_step_stats;

/* Creates a simulation.  grid: cells per axis; patch: P (power of two,
 * P/2^levels >= 2 for BL5/3); levels: L >= 1; eps: threshold constant c of
 * Sec. 2.2 (0 = lossless up to rounding).  Allocates all device memory.
 * Returns WCS_E_UNSUPPORTED if no kernel was compiled for the combination
 * (scheme, wavelet, compute, detail_store, P, L).  patch = 0 and/or
 * levels = 0: chosen by the patch autotuner (wcs_autotune) in
 * wcs_init_macro, on the caller's initial fields, among the compiled
 * kernels of the configuration whose P divides every axis (and that match
 * the non-zero one); nothing is allocated before, the simulation must then
 * start from wcs_init_macro, and wcs_patch_config tells the choice.
 * WCS_E_UNSUPPORTED if no compiled kernel fits. */
wcs_status wcs_create_sim(const wcs_grid* grid, int scheme, int patch, int levels, double eps,
                          const wcs_opts* opts, wcs_sim** out);

/* The simulation's patch size and levels (0 while a choice deferred to
 * wcs_init_macro is pending). */
wcs_status wcs_patch_config(const wcs_sim* sim, int* patch, int* levels);

/* Frees everything the simulation holds.  NULL is accepted. */
void wcs_destroy(wcs_sim* sim);

/* Initial state from macroscopic fields, each a dense array of doubles laid
 * out [ny][nx] over the unique nodes (nx = n[0] cells, or n[0]+1 nodes on a
 * non-periodic BL5/3 axis), x fastest.  D2Q9: (rho, u_x, u_y), the state is
 * the equilibrium.  D3Q19: (rho, u_x, u_y, u_z) laid out [nz][ny][nx], the
 * equilibrium.  EULER2D: (rho, u, v, p).  TRANSPORT: (W).  SWE: (h, u, v).  fields[k] are host pointers if
 * src_is_device == 0, else device pointers.  Encodes state 0. */
wcs_status wcs_init_macro(wcs_sim* sim, const double* const* fields, int nfields, int src_is_device);

/* Advances n time steps (one fused kernel launch each, enqueued on the
 * simulation's stream; does not synchronise). */
wcs_status wcs_step(wcs_sim* sim, int64_t n);

/* Waits for the stream and returns the sticky device status as a status. */
wcs_status wcs_sync(wcs_sim* sim);

/* Decodes the current state of one field (D2Q9/D3Q19: population i;
 * EULER2D: 0..3) into a dense [ny][nx] ([nz][ny][nx] in 3-D) array over the
 * unique nodes.  dtype: 0 = double,
 * 1 = float.  dst is a device pointer if dst_is_device, else host.
 * field = -1 writes every field, one after the other. */
wcs_status wcs_export_field(wcs_sim* sim, int field, void* dst, int dst_is_device, int dtype);

/* Bytes of device memory that hold the compressed state: the records of
 * the current state plus the ghost ring it needs (none for 2-D BL5/3
 * patches, which decode their ghosts from the neighbours' records) and
 * the patch table. */
int64_t wcs_compressed_bytes(const wcs_sim* sim);

/* Every byte of device memory the simulation holds: both record arenas at
 * their capacity, rings, tables, control block, FP64 sums and (3-D) the
 * per-SM scratch.  -1 for NULL. */
int64_t wcs_resident_bytes(const wcs_sim* sim);

/* Replaces the current state by dense values over the unique nodes (the
 * layout of wcs_export_field: field = -1 takes F planes one after the
 * other, else one field's plane) and encodes it again (threshold, quantise,
 * records, ghost rings where kept, FP64 sums and, EULER2D and SWE, the signal speed for the
 * next step); the step count and time are kept.  dtype 0 = double, 1 =
 * float, rounded to the compute type; src is a device pointer if
 * src_is_device, else host.  Used to start from a given state, or to hand a
 * state decoded elsewhere to the library (field = -1 also initialises a
 * fresh simulation).  Takes one uncompressed copy of the state as temporary
 * device memory (one field: the other fields are decoded into it first).
 * Synchronises. */
wcs_status wcs_import_field(wcs_sim* sim, int field, const void* src, int src_is_device, int dtype);

/* Entropy-codes the records of the current state: the library's own
 * lossless stage on top of the bitmask codec, where the paper (Sec. 2.3.2)
 * runs a general-purpose byte compressor.  Order-0 byte-wise rANS (range
 * asymmetric numeral systems) with one frequency table for the state,
 * scaled to 2^12; layout: u32 npatch, u32 12, u16 freq[256], per patch u32
 * record bytes and u32 coded bytes, then the patches' streams (each: the
 * final 32-bit coder state, little endian, then its renormalisation bytes
 * in decoding order).  The coded state is decoded again on the device and
 * compared byte for byte with the records (a difference returns
 * WCS_E_CUDA).  dst_host = NULL asks for the size only (*nbytes); a buffer
 * of cap < *nbytes bytes gets WCS_E_ARG.  Synchronises; takes temporary
 * device memory of about 1.5x the live record bytes. */
wcs_status wcs_entropy_code(wcs_sim* sim, void* dst_host, int64_t cap, int64_t* nbytes);

/* FP64 diagnostics of the current state (synchronises). */
wcs_status wcs_stats(wcs_sim* sim, wcs_step_stats* out);
/* The same without a synchronisation: wcs_stats_enqueue queues, on the
 * simulation's stream behind the work already enqueued, a copy of the
 * control block and of the per-patch FP64 sums into slot `slot` (0..3) of
 * pinned host memory that the library owns (allocated at the first call:
 * 4 x (npatch x F x 8 + 88) bytes); wcs_stats_collect waits for that copy
 * and fills out exactly as wcs_stats would have for that step (same sums,
 * same order).  A slot is free again after its collect; collecting an
 * empty slot is WCS_E_ARG.  No arena-overflow recovery here: a failed step
 * shows in out->status, and wcs_sync recovers or reports it. */
wcs_status wcs_stats_enqueue(wcs_sim* sim, int slot);
wcs_status wcs_stats_collect(wcs_sim* sim, int slot, wcs_step_stats* out);

/* Detail coefficients kept in the current state (the survivors of the
 * threshold, all patches and fields; coarse samples not counted), counted
 * on the device from the records' tables.  Synchronises; -1 on error. */
int64_t wcs_survivors(wcs_sim* sim);

/* hi + lo coarse storage (opts.coarse_hilo): copies the lo parts of the
 * current state into the host buffer out, npatch x nfields x NC1^dims
 * floats (patch-major, then field, then coarse sample iy NC1 + ix, or
 * (iz NC1 + iy) NC1 + ix in 3-D, with NC1 = P/2^L + 1), n = their count.  Synchronises the stream.  WCS_E_ARG if
 * the option is off, before the init, or for a wrong n. */
wcs_status wcs_coarse_lo(wcs_sim* sim, float* out, int64_t n);

/* Copies the record of one patch of the current state (the byte format of
 * the oracle) to host memory.  *nbytes receives its size; if cap is too
 * small nothing is copied and WCS_E_ARG is returned.  A record holds at
 * most 16 MiB - 1 bytes (the patch table packs offset << 24 | size); a
 * larger one is reported as WCS_E_ARENA_FULL (P = 64 with 9 FP32 fields
 * needs at most ~160 KB). */
wcs_status wcs_export_record(wcs_sim* sim, int64_t patch, void* dst, int64_t cap, int64_t* nbytes);

/* Export without device allocation.  Same result as wcs_export_field with a
 * host destination, for callers that cannot call cudaMalloc at that point:
 * a process whose device memory is already taken up by its simulations (the
 * temporary buffer of wcs_export_field could fail with WCS_E_OOM), or a
 * latency-bound loop that must not pay for cudaMalloc/cudaFree and the
 * device-wide synchronisation they imply.  The paper has no counterpart.
 *
 * The decoded field is staged in one library-wide device array of
 * WCS_NOALLOC_SCRATCH_BYTES bytes, reserved on every GPU that loads the
 * library until the process exits, then copied to host_dst (caller-owned,
 * ny*nx values of the given dtype; field = -1 writes every field).  Requests
 * larger than the array return WCS_E_ARG with a message saying so.  The
 * first call on a device looks the array's device address up (with that
 * device current); make that first call before any CUDA stream capture.
 * Every call shares the array and overwrites it completely for the range it
 * exports; calls whose work overlaps on the GPU (several simulations on
 * different streams or host threads) race on it and must be serialised by
 * the caller.  The simulation's device must be the current device (else
 * WCS_E_ARG).  Synchronises the simulation's stream; allocates nothing. */
#define WCS_NOALLOC_SCRATCH_BYTES (16u << 20)
wcs_status wcs_export_field_noalloc(wcs_sim* sim, int field, void* host_dst, int dtype);

/* Number of patches and fields, dense node counts. */
wcs_status wcs_shape(const wcs_sim* sim, int64_t* npatch, int* nfields, int64_t* nodes_x, int64_t* nodes_y);
/* The same with the node counts of all three axes (nodes[2] = 1 in 2-D). */
wcs_status wcs_shape3(const wcs_sim* sim, int64_t* npatch, int* nfields, int64_t* nodes);

/* Per-launch device time of the last wcs_step kernels is not tracked here;
 * callers time with events on the stream.  This returns the stream. */
void* wcs_stream(const wcs_sim* sim);

/* Last error message of the simulation (or of the last failed create when
 * sim is NULL).  Valid until the next call on the same simulation. */
const char* wcs_last_error(const wcs_sim* sim);

/* ------------------------------------------------------------------------
 * Batches of independent simulations (many grids of different sizes; one
 * launch per step when the batch holds the two patch sizes of a merged
 * kernel (D2Q9, BL5/3, FP32 compute, BF16 or FP32 details: 64 cells / 4
 * levels with 32 / 3), else
 * one launch per kind of kernel; six steps captured in one CUDA graph and
 * replayed).  Every simulation must be initialised, created on the same
 * stream and at the same step; 3-D simulations and simulations with a
 * learned threshold are stepped alone (WCS_E_UNSUPPORTED).  The batch borrows the simulations (destroy
 * the batch before them); stepping one of them outside the batch makes the
 * next wcs_batch_step fail with WCS_E_ARG.
 * ---------------------------------------------------------------------- */
typedef struct wcs_batch wcs_batch;
wcs_status wcs_batch_create(wcs_sim* const* sims, int nsims, wcs_batch** out);
void wcs_batch_destroy(wcs_batch* b);
/* Advances every simulation of the batch by n steps (asynchronous). */
wcs_status wcs_batch_step(wcs_batch* b, int64_t n);
/* Waits and returns the first device error of any simulation.  Arenas:
 * a simulation with automatic arenas gets room for its records to double
 * when the batch is created (the batch holds its arena pointers, so they
 * are not resized while it steps); one whose records outgrew them all the
 * same froze at the input of the failed step, and this call re-runs its
 * lost steps alone with doubled arenas (counted in arena_reruns) and
 * updates the batch, so that every simulation is at the batch's step
 * again.  Fixed arenas (arena_factor > 0) report WCS_E_ARENA_FULL. */
wcs_status wcs_batch_sync(wcs_batch* b);
/* Kernel launches per step (1 when the batch's two patch sizes run in one
 * merged persistent launch, else one per kind of kernel) and the merged
 * launch's grid (0 if none). */
wcs_status wcs_batch_launches_per_step(const wcs_batch* b, int* launches, int* grid);
/* Launch-shape tuner of a merged batch: times `steps` steps with each of the
 * ncand grids (blocks of the persistent launch; more blocks than items are
 * cut to the items) and keeps the fastest; per-step times to ms_per_step
 * (may be NULL).  The simulations advance by ncand x steps steps.
 * WCS_E_UNSUPPORTED if the batch has no merged launch. */
wcs_status wcs_batch_tune_launch(wcs_batch* b, const int* grids, int ncand, int steps, double* ms_per_step);
const char* wcs_batch_last_error(const wcs_batch* b);

/* Patch-size autotuner (2-D and D3Q19): for each candidate (P[i], levels L[i]) creates a
 * simulation on the caller's initial fields (layout of wcs_init_macro),
 * times `steps` steps with CUDA events and writes the index of the fastest
 * to *best (and the per-step times to ms_per_step[ncand] if not NULL).
 * Candidates without a compiled kernel are skipped.  Results are cached for
 * the process per (grid, scheme, options, eps, candidate list). */
wcs_status wcs_autotune(const wcs_grid* grid, int scheme, const wcs_opts* opts, double eps, const int* P, const int* L,
                        int ncand, const double* const* fields, int nfields, int src_is_device, int steps, int* best,
                        double* ms_per_step);

/* ------------------------------------------------------------------------
 * Learned per-patch threshold (not in the paper, which uses one constant c):
 * a network in -> 64 -> 64 -> 1 (GELU, FP32) maps per-patch features to
 * log10(eps).  Features of a patch: its detail nodes are grouped by (l, S),
 * l = the largest per-axis class of the node, S = the axes of that class
 * (x, y or both); per group, over all fields, log10(mean d^2 + 1e-30) and
 * log10(max |d| + 1e-30) of the forward-transformed patch before the
 * threshold; groups in the order l = 1..L, S = x, y, xy, so in = 6L.
 * Label: log10 of the largest eps = 10^(-7 + k/8), k = 0..40, whose
 * thresholding (constant rule, no quantisation) changes the patch by at
 * most delta * ||patch||_2 after the inverse transform, refined by four
 * bisections in log eps (steps under 2%); -7 if none passes, -2 if all do.
 * ---------------------------------------------------------------------- */
typedef struct wcs_mlp wcs_mlp;
/* Features and labels of every patch of a dense FP32 state [F][ny][nx]
 * (device; periodic axes), FP64 arithmetic, patches in row order
 * (pid = py * (nx / patch) + px).  feat_dev: npatch x 6L floats, label_dev:
 * npatch floats (log10 eps).  levels <= 8; (patch + 1)^2 FP64 values x 3 must
 * fit in shared memory (patch <= 96); else WCS_E_UNSUPPORTED. */
wcs_status wcs_features_labels(const float* dense_dev, int nfields, int64_t nx, int64_t ny, int wavelet, int patch,
                               int levels, double delta, float* feat_dev, float* label_dev, void* stream);
/* The same for cubic BL5/3 patches of a periodic 3-D state [F][nz][ny][nx]
 * (the D3Q19 geometry; patch 32 or 16, levels 3): 7 axis sets per level, so
 * npatch x 42 features; the transforms run in FP32 like the 3-D step, the
 * threshold test and the error sums in FP64.  Patches in the order
 * pid = (pz * npy + py) * npx + px.  Synchronises the stream; allocates a
 * scratch of F (patch+1)^3 floats per SM for the call. */
wcs_status wcs_features_labels3(const float* dense_dev, int nfields, int64_t nx, int64_t ny, int64_t nz, int patch,
                                int levels, double delta, float* feat_dev, float* label_dev, void* stream);
wcs_status wcs_mlp_create(int nin, wcs_mlp** out);
void wcs_mlp_destroy(wcs_mlp* m);
int wcs_mlp_nparam(const wcs_mlp* m);
/* parameters: W1[64][in], b1[64], W2[64][64], b2[64], W3[64], b3 (host) */
wcs_status wcs_mlp_set_weights(wcs_mlp* m, const float* w_host);
wcs_status wcs_mlp_get_weights(const wcs_mlp* m, float* w_host);
/* mean squared error of the outputs against t on n samples and its gradient */
wcs_status wcs_mlp_grad(wcs_mlp* m, const float* X_dev, const float* t_dev, int n, float* grad_host, float* loss_host);
/* Adam (lr, 0.9, 0.999) over minibatches: batches_host holds epochs x
 * (n / batch) x batch sample indices; loss of the last minibatch of each
 * epoch to loss_history_host[epochs]. */
wcs_status wcs_mlp_train(wcs_mlp* m, const float* X_dev, const float* t_dev, int n, const int* batches_host, int epochs,
                         int batch, float lr, float* loss_history_host);
/* Trains on raw features: the per-input mean and sample deviation of X_dev
 * (n x nin, device, FP64 sums) and the mean of t_dev are taken on the device;
 * the output bias starts at the mean target (Adam restarted); training
 * (as wcs_mlp_train, same batches_host layout) runs on the standardised
 * copy (x - mean) / max(deviation, sd_floor); the standardisation is then
 * folded into the first layer (W1 / sd, b1 - (W1 / sd) mean), so that the
 * network takes the raw features a learned-mode step writes.  n >= 2,
 * sd_floor > 0.  stats_host (optional, 2 (nin + 1) doubles): mean and
 * deviation of each input, then of t.  Allocates n x nin floats of scratch
 * for the call; synchronises. */
wcs_status wcs_mlp_fit(wcs_mlp* m, const float* X_dev, const float* t_dev, int n, const int* batches_host, int epochs,
                       int batch, float lr, double sd_floor, float* loss_history_host, double* stats_host);
wcs_status wcs_mlp_forward(wcs_mlp* m, const float* X_dev, int n, float* y_dev);
/* per-patch eps = clamp(10^network(features), lo, hi); non-finite -> fallback */
wcs_status wcs_mlp_eps(wcs_mlp* m, const float* feat_dev, int n, double lo, double hi, double fallback, double* eps_dev,
                       void* stream);
/* Every following step of the simulation writes the features of its new
 * state and sets each patch's eps for the next step from the network
 * (patch edge lines keep the uniform eps so that shared nodes stay
 * identical).  m = NULL returns to the uniform eps. */
wcs_status wcs_sim_use_mlp(wcs_sim* sim, wcs_mlp* m, double eps_lo, double eps_hi);
/* Sets the threshold constant of every patch (host array of npatch values,
 * edge lines keep the uniform eps); NULL returns to the uniform eps. */
wcs_status wcs_sim_set_patch_eps(wcs_sim* sim, const double* eps_host);
/* current per-patch features (npatch x 6L) and eps (npatch), host copies */
wcs_status wcs_sim_patch_data(wcs_sim* sim, float* feat_host, double* eps_host);

/* ------------------------------------------------------------------------
 * Uncompressed baseline (the "uncompressed" side of the metric): the same
 * scheme on dense FP32 arrays, two lattices, one kernel per step.
 * ---------------------------------------------------------------------- */
typedef struct wcs_dense wcs_dense;

wcs_status wcs_dense_create(const wcs_grid* grid, int scheme, const wcs_opts* opts, wcs_dense** out);
void wcs_dense_destroy(wcs_dense* d);
wcs_status wcs_dense_init_macro(wcs_dense* d, const double* const* fields, int nfields, int src_is_device);
wcs_status wcs_dense_step(wcs_dense* d, int64_t n);
wcs_status wcs_dense_export_field(wcs_dense* d, int field, void* dst, int dst_is_device, int dtype);
int64_t wcs_dense_bytes(const wcs_dense* d);

#ifdef __cplusplus
}
#endif
#endif /* WCSIM_H */
