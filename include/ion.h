/*
 * ion.h -- C ABI of the GB300 InfOli network simulator (libion.so).
 *
 * The library advances networks of three-compartment inferior-olive cells coupled by
 * dendritic gap junctions, one synchronous explicit-Euler step at a time, on one GPU.
 * Paper: Smaragdos et al., "BrainFrame: a node-level heterogeneous accelerator
 * platform for neuron simulations" (arXiv 1612.01501):
 *   - Sec. 2.2 "The InfOli Workload": a new cell state depends only on the cell's
 *     previous state, the previous dendritic voltages of its gap-junction partners and
 *     the evoked input; compartments and gap junctions are updated concurrently with a
 *     fixed 50 us step.  Table "reqs": 19 state words, 20 conductances, 1 evoked input
 *     and 1 connectivity word per connection per cell.
 *   - Algorithm 1 (RGJ): Ic_i += w_ij (0.8 e^{-dV^2/100} + 0.2) dV, dV = V_dend,i - V_dend,j.
 *   - Sec. 2.3: connectivity is a user-programmed weight matrix; here either one
 *     uniform weight for every pair (dense all-to-all) or a CSR matrix.
 *   - Sec. 2.4.3: states and evoked inputs are copied to the device once before the
 *     run; no host data is needed while it runs.
 *
 * Conventions for every entry point:
 *   - Each call returns an ion_status and never aborts or exits the process.
 *   - Host buffers passed in are copied before the call returns; the caller keeps
 *     ownership.  Buffers marked ION_DEVICE are read in place (borrowed) and must stay
 *     valid for as long as the documentation of the argument says.
 *   - Work is enqueued on the CUDA stream given in ion_params.cuda_stream (NULL: a
 *     non-blocking stream the handle creates and owns).  ion_step is asynchronous; errors the device detects
 *     (a non-finite state, a barrier that timed out) are sticky and are returned by
 *     the next ion_sync / ion_read_* call.
 *   - A handle is used by one host thread at a time.
 *   - Units: mV, ms, mS/cm^2, uF/cm^2, uA/cm^2; [Ca] in the model's units.
 *   - State is structure-of-arrays: field f of cell i is element f * n_cells + i of a
 *     full-state buffer, fields in the order of enum ion_field.
 */
#ifndef ION_H
#define ION_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ION_NFIELDS 19 /* Table "reqs": 19 state words per cell */
#define ION_NPARAMS 25 /* model constants, order of enum ion_param */
#define ION_NGATES 12  /* gating variables with a rate function */
#define ION_NCELLPARAMS 20 /* per-cell model constants: entries 0..19 of enum ion_param */

typedef enum {
    ION_OK = 0,
    ION_ERR_INVALID_ARG = 1, /* a NULL pointer, a size out of range, an unknown enum   */
    ION_ERR_BAD_CSR = 2,     /* CSR not monotone, index out of range, self loop,
                                unsorted row, or not symmetric                          */
    ION_ERR_OOM = 3,         /* device or host allocation failed                       */
    ION_ERR_CUDA = 4,        /* a CUDA runtime call failed (see ion_last_error)        */
    ION_ERR_NONFINITE = 5,   /* the device saw a NaN or Inf in a voltage or [Ca]       */
    ION_ERR_TIMEOUT = 6,     /* a bounded device wait (grid barrier) gave up           */
    ION_ERR_UNSUPPORTED = 7  /* valid request this build does not handle               */
} ion_status;

/* State fields (Table "reqs": 19 words).  m_s, m_a, I_CaH and I_c hold the values used
 * during the last step (they are outputs, never read back by the update); g_CaL is a
 * per-cell constant. */
enum ion_field {
    ION_V_DEND = 0, ION_V_SOMA, ION_V_AXON, ION_CA,
    ION_R, ION_S, ION_Q,                         /* dendrite gates              */
    ION_K, ION_L, ION_M_S, ION_H_S, ION_N_S, ION_X_S, /* soma gates             */
    ION_M_A, ION_H_A, ION_X_A,                   /* axon gates                  */
    ION_G_CAL, ION_I_CAH, ION_I_C,
    ION_FIELD_ALL = -1                           /* all 19 fields, SoA order    */
};

/* Model constants.  Entries 0..19 are the per-cell constants a neuron may own (see
 * ion_params.cell_params): 13 conductances (g_int and the 12 channel conductances), the two
 * area ratios p1, p2 and five reversal potentials.  Table "reqs" counts 20 conductances per
 * neuron; the three-compartment model used here has 13. */
enum ion_param {
    ION_P_GINT = 0, ION_P_P1, ION_P_P2,
    ION_P_GCAH, ION_P_GKCA, ION_P_GH, ION_P_GLD,
    ION_P_GCAL, ION_P_GNAS, ION_P_GKDRS, ION_P_GKS, ION_P_GLS,
    ION_P_GNAA, ION_P_GKA, ION_P_GLA,
    ION_P_VNA, ION_P_VK, ION_P_VCA, ION_P_VH, ION_P_VL,
    ION_P_CM, ION_P_CA_IN, ION_P_CA_OUT, ION_P_V0, ION_P_CA0
};

enum ion_net_kind {
    ION_DENSE_UNIFORM = 0, /* all-to-all, one weight g_c for every pair (RGJ, C = 100 %) */
    ION_CSR = 1,           /* CSR weight matrix (RGJ at any density)                     */
    ION_NO_GJ = 2,         /* independent cells (NGJ use case, Sec. 2.3.3)               */
    ION_DENSE_MATRIX = 3   /* all-to-all with an N x N weight matrix (every pair stored)   */
};
enum ion_mem { ION_HOST = 0, ION_DEVICE = 1 };

enum ion_flag {
    ION_FLAG_KAHAN = 1u << 0,      /* compensated dense gap-junction sums (default on)     */
    ION_FLAG_PERSISTENT = 1u << 1, /* dense: one cooperative launch per ion_step call, state in
                                      registers, a bounded grid barrier per step (if every CTA
                                      fits on the GPU at once; else per-step launches)       */
    ION_FLAG_SURROGATE = 1u << 2,  /* MLP surrogate for the channel rate functions         */
    ION_FLAG_CHECKS = 1u << 3,     /* non-finite scan of every cell every check_every steps */
    ION_FLAG_NO_GRAPH = 1u << 4,   /* launch steps directly instead of CUDA-graph replay    */
    ION_FLAG_SPLIT = 1u << 5,      /* separate gap-junction and cell-update kernels         */
    ION_FLAG_HALF_WORK = 1u << 6,  /* evaluate each unordered pair once (I_ij = -I_ji).  Dense,
                                      with PERSISTENT and several CTAs: column sums exchanged
                                      through L2 (two bounded barriers per step).  CSR (host
                                      arrays, symmetric weights): the upper triangle only,
                                      each mirrored term through a per-edge slot, then a
                                      fixed-order gather per row (two launches per step; not
                                      with SPLIT, SGJ, PERSISTENT or SURROGATE)            */
    ION_FLAG_CSR_AS_GIVEN = 1u << 7, /* CSR: keep 32-bit columns and per-edge weights even when
                                      a compact layout applies (see ion_csr_layout)         */
    ION_FLAG_SGJ = 1u << 8,        /* SGJ use case (Sec. 2.3.2): each connection contributes
                                      w (V_i - V_j) instead of the RGJ term.  Dense or CSR;
                                      not with PERSISTENT, SURROGATE, SPLIT or batches      */
    ION_FLAG_SURROGATE_WARP_MMA = 1u << 10, /* with SURROGATE: run the MLP on warp-level
                                      mma.sync (m16n8k16) instead of tcgen05 with TMEM
                                      accumulators (kept for comparison)                   */
    ION_FLAG_NO_PDL = 1u << 9      /* launch the per-step kernels as ordinary stream-ordered
                                      launches.  By default each is launched with programmatic
                                      stream serialization: its CTAs may be scheduled while the
                                      previous step's kernel drains, and wait on the device
                                      (griddepcontrol.wait) for its completion before touching
                                      memory.  Results are identical either way.             */
};

typedef struct {
    int32_t n_cells; /* >= 1 */
    int32_t kind;    /* enum ion_net_kind */
} ion_net;

/* Connectivity.  Dense: g_c is the weight of every pair.  Dense matrix: weight[n * n]
 * (row-major, W[i][j] weighs the current into cell i from cell j; the diagonal pair
 * contributes zero whatever its weight); row_ptr/col_idx unused; the matrix is copied into
 * the handle (padded rows), host matrices are checked to be finite.  CSR: row_ptr[n+1] (int32,
 * row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz), col_idx[nnz] in [0, n), strictly
 * ascending within a row, no self loops, pattern symmetric; weight[nnz] (may be NULL:
 * every weight is g_c).  mem says where the three arrays live; ION_DEVICE arrays are
 * borrowed and must outlive the handle.  The symmetry check is done for host arrays
 * only (device arrays are trusted). */
typedef struct {
    float g_c;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const float *weight;
    int64_t nnz;
    int32_t mem;
} ion_conn;

typedef struct {
    double v[ION_NPARAMS];
} ion_model;

typedef struct {
    double dt_ms;               /* 0 means 0.05 (the paper's 50 us step)                  */
    const ion_model *model;     /* NULL means ion_model_default()                         */
    uint32_t flags;             /* enum ion_flag                                          */
    const void *surrogate;      /* ion_surrogate_weights* when ION_FLAG_SURROGATE          */
    int32_t check_every;        /* steps between non-finite scans (0 = 64)                */
    int32_t graph_steps;        /* steps captured per CUDA graph (0 = 50)                 */
    uint64_t barrier_timeout_ns;/* bound on a persistent kernel's grid barrier (0 = 2 s)  */
    void *cuda_stream;          /* cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream;
                                   NULL: the handle creates and owns a non-blocking stream  */
    const void *tune;           /* ion_tune* launch shape override, NULL = built-in choice */
    int64_t debug_delay_ns;     /* test hook, 0 in production: with ION_FLAG_PERSISTENT one CTA
                                   sleeps this long before its first grid barrier (a short
                                   barrier_timeout_ns then yields ION_ERR_TIMEOUT)          */
    const float *cell_params;   /* per-cell model constants (Table "reqs": every neuron has its
                                   own conductances), or NULL for the model table's values in
                                   every cell.  Host FP32 array of ION_NCELLPARAMS x n_cells,
                                   structure of arrays: entry p of cell i at p * n_cells + i,
                                   p in enum ion_param order (g_int, p1, p2, the 12 channel
                                   conductances, V_Na, V_K, V_Ca, V_h, V_L).  Copied at
                                   creation; checked finite, 0 < p1, p2 < 1.  Entry ION_P_GCAL
                                   is not read: g_CaL is per cell already (state field
                                   ION_G_CAL).  Dense uniform, CSR and NO_GJ networks only; with
                                   gap junctions the currents and the cell update then run as
                                   two launches per step (as ION_FLAG_SPLIT).  Not with
                                   PERSISTENT, SURROGATE, SGJ, a dense matrix or batches
                                   (ION_ERR_UNSUPPORTED)                                   */
    uint32_t debug_barrier_base;/* test hook, 0 in production: the value the grid-barrier
                                   arrival counter of a persistent launch starts from, so that
                                   a test can make it wrap past 2^32 within a few steps     */
} ion_params;

/* Evoked input (Sec. 2.2: one evoked-input word per cell per step).
 *   ION_INPUT_NONE   -- no evoked current;
 *   ION_INPUT_PULSES -- I_app(t, i) = sum of amp[p] over pulses p with cell[p] == i and
 *                       t_begin[p] <= t < t_end[p] (t = absolute step index);
 *   ION_INPUT_DENSE  -- I_app(t, i) = dense[(t - t_first) * n_cells + i] for the
 *                       n_steps of one ion_step call (t_first = its first step). */
enum ion_input_kind { ION_INPUT_NONE = 0, ION_INPUT_PULSES = 1, ION_INPUT_DENSE = 2 };
typedef struct {
    int32_t kind;
    int32_t mem;           /* where dense / pulse arrays live                        */
    const float *dense;    /* [n_steps x n_cells], row-major                          */
    int32_t n_pulses;
    const int32_t *pulse_cell;
    const int64_t *pulse_begin;
    const int64_t *pulse_end;
    const float *pulse_amp;
} ion_input;

/* Launch-shape override (filled by ion_autotune, or by hand).  0 = the built-in choice. */
typedef struct {
    int32_t dense_rows_per_warp; /* R: 1, 2, 4, 6 or 8 (batches: 1, 2, 4 or 8)      */
    int32_t dense_warps;         /* W warps per CTA (<= 1024 threads for R <= 2,
                                    768 otherwise), a multiple of dense_col_splits */
    int32_t dense_col_splits;    /* GJ: 1, 2 or 4 warps share a row group, each
                                    taking every GJ-th group of 128 columns         */
    int32_t csr_lanes_per_row;   /* 1, 2, 4, 8, 16 or 32                            */
    int32_t csr_rows_per_cta;    /* rows per CTA of 256 threads, 1..256             */
    int32_t csr_lanes_scale;     /* batches: 0 = lanes per row from each network's
                                    mean degree, +1 = twice that, -1 = half        */
    int32_t csr_staging;         /* single CSR networks: 0 = choose (stage when the
                                    mean degree is 64 or more and at least 32 per
                                    chunk, or the CSR exceeds 96 MB), 1 = gather V_dend
                                    through L1/L2, 2 = stage V_dend in shared memory
                                    128 KB at a time (one CTA per SM)                */
    int32_t csr_bank_order;      /* single CSR networks with equal weights: 1 = store the
                                    16-bit columns in shared-memory bank order (see
                                    ion_csr_bank_order); 0 = as sorted.  Read at creation */
} ion_tune;

typedef struct ion_sim ion_sim;

/* ---- model -------------------------------------------------------------------- */

/* The library's constants table (its own copy; the oracle keeps another). */
void ion_model_default(ion_model *out);

/* Every gate's steady state and time constant at voltage V and calcium ca, FP32, as
 * the device computes them (gate order: r s q k l m_s h_s n_s x_s m_a h_a x_a; tau of
 * the instantaneous m_s, m_a is 0).  xinf and tau are host arrays of 12 floats each. */
ion_status ion_rates(float V, float ca, float *xinf, float *tau);

/* Default initial state of n cells into host buffer out[19 * n] (FP32, SoA): every
 * compartment at V_0, each gate at its steady state there, [Ca] at [Ca]_0. */
ion_status ion_default_state(const ion_model *model, int32_t n, float *out);

/* ---- simulation handle -------------------------------------------------------- */

/* Validate, copy to the device and prepare launches of one network.
 * init_state: host FP32 buffer of 19 * n_cells values (SoA) or NULL for the default.
 * On success *out owns device memory until ion_destroy. */
ion_status ion_create(const ion_net *net, const ion_conn *conn, const ion_params *params,
                      const float *init_state, ion_sim **out);

/* Several independent networks advanced together: one launch per time step covers all
 * of them (a list of tiles, each one network's rows), and ion_step replays CUDA graphs of
 * graph_steps launches.  Cells are numbered consecutively across networks (network b's
 * cell i is global cell offset_b + i, offset_b = n_0 + ... + n_{b-1}); init_state, the
 * state read and written, pulse cells and trace samples all use this numbering.
 * Dense networks may have at most 8192 cells; CSR arrays must be host memory.
 * ION_FLAG_PERSISTENT: each ion_step call is one cooperative launch (replayed from a CUDA
 * graph) that advances every network by all its steps.  The networks are cut into pieces
 * of at most 256 rows, dealt out to CTAs that are all resident at once; a piece waits
 * (bounded by barrier_timeout_ns, then ION_ERR_TIMEOUT) only until every piece of its own
 * network has finished the previous step, so there is no grid-wide barrier.  The states
 * equal those of the per-step launches bit for bit.  Dense evoked input (ION_INPUT_DENSE)
 * falls back to per-step launches; not with ION_FLAG_CSR_AS_GIVEN.
 * ION_FLAG_SPLIT, ION_FLAG_SGJ and ION_FLAG_SURROGATE are not supported here. */
ion_status ion_create_batch(int32_t n_nets, const ion_net *nets, const ion_conn *conns,
                            const ion_params *params, const float *init_state,
                            ion_sim **out);

/* Install the evoked input used by later ion_step calls that pass NULL.  Pulse arrays
 * are copied; a DENSE input cannot be installed. */
ion_status ion_set_input(ion_sim *sim, const ion_input *input);

/* Advance n_steps >= 0 steps on the handle's stream (asynchronous).  input NULL uses
 * the installed input; a DENSE input must hold n_steps x n_cells values and, if it is
 * ION_DEVICE, stay valid until the stream reaches the end of this call's work. */
ion_status ion_step(ion_sim *sim, int64_t n_steps, const ion_input *input);

/* Wait for the handle's stream, then report any sticky device error. */
ion_status ion_sync(ion_sim *sim);

/* Copy state to host memory `out` (count floats: n_cells for one field, 19 * n_cells
 * for ION_FIELD_ALL).  Synchronises; returns a sticky device error if there is one
 * (the copy is still made). */
ion_status ion_read_state(ion_sim *sim, int32_t field, float *out, int64_t count);

/* Overwrite state from host memory `in` (same sizes as ion_read_state).  Ordered on
 * the handle's stream after earlier steps. */
ion_status ion_write_state(ion_sim *sim, int32_t field, const float *in, int64_t count);

/* Device pointer of one field of the current state (valid until the next ion_step).
 * Not available for batches (their state is laid out in padded segments). */
ion_status ion_state_device_ptr(ion_sim *sim, int32_t field, float **out);

/* Record V_axon of every cell every `stride` steps into a device ring of `capacity`
 * samples (0 disables); ion_read_trace copies the samples recorded since the last read
 * (oldest first) to host memory: out[s * n_cells + i]. */
ion_status ion_set_trace(ion_sim *sim, int32_t stride, int32_t capacity);
ion_status ion_read_trace(ion_sim *sim, float *out, int64_t max_samples, int64_t *n_written);

/* Asynchronous form of ion_read_trace (Sec. 2.4.3: the transfer of step t overlaps the
 * computation of step t + 1): queues, on the handle's own copy stream and after the steps
 * already enqueued, the copy of the samples recorded since the last read (oldest first,
 * out[s * n_cells + i]) and returns at once with *n_queued.  `out` must stay valid until
 * ion_trace_wait (or ion_destroy) returns; pinned host memory lets the copy overlap the
 * steps that follow.  Later steps that would overwrite a ring slot the copy still reads
 * wait for it on the device.  Not for batches (ION_ERR_UNSUPPORTED). */
ion_status ion_read_trace_async(ion_sim *sim, float *out, int64_t max_samples, int64_t *n_queued);
/* Block until the last queued trace copy has landed in host memory. */
ion_status ion_trace_wait(ion_sim *sim);

/* Time candidate launch shapes on this handle's own network(s), `steps` time steps each,
 * and keep the fastest (the state and step count are restored afterwards).  Single
 * dense networks: (R, W, GJ) near the cost model's optimum; single CSR networks: lanes
 * per row and rows per CTA around the degree-based choice; batches: rows per dense tile,
 * rows per CSR tile and the lanes-per-row scale.  *chosen (nullable) receives the table.
 * Not for ION_FLAG_PERSISTENT handles.  Synchronises. */
ion_status ion_autotune(ion_sim *sim, int32_t steps, ion_tune *chosen);

/* Storage the handle streams per stored edge of a CSR network (host-copied CSR only; a
 * borrowed device CSR is used as given):
 *   *index_bytes  2 when every column is kept as its low 16 bits and used: V_dend is
 *                 staged in shared memory in chunks of 32 768 cells (the column relative to
 *                 its chunk fits in 16 bits), or the network has at most 65 536 cells and a
 *                 mean degree of at least 32; else 4;
 *   *weight_bytes 0 when every weight is bitwise equal (one scalar is kept), else 4;
 *   *staged       1 when V_dend is staged in shared memory chunk by chunk, else 0.  A
 *                 staged handle also keeps its columns chunk by chunk, each row's segment
 *                 padded to a multiple of 8 with entries that pair the row with itself
 *                 (dV = 0: they add exactly 0); the figures above count the stored edges.
 * Both compactions are exact: the kernels evaluate the same edges with the same values.
 * ION_FLAG_CSR_AS_GIVEN turns them off.  Dense / NGJ handles report 0, 0, 0.  Any output
 * pointer may be NULL. */
ion_status ion_csr_layout(const ion_sim *sim, int32_t *index_bytes, int32_t *weight_bytes, int32_t *staged);

/* Edge order for the shared-memory gathers of the staged CSR kernel (host only, no device
 * call).  The kernel reads the 16-byte-aligned body of each row's per-chunk segment
 * (columns in [c chunk, (c + 1) chunk)) as groups of eight edges, lane l of a row taking
 * groups l, l + lanes, ...; one gather reads position k of one round of groups, and its
 * shared-memory banks are the columns mod 32.  perm[e] (nnz = row_ptr[n] entries, caller
 * owned) receives the original index of the edge to place at position e: a permutation
 * within each segment's body that gives every gather set distinct banks where the row
 * allows it (heads and tails keep their order).  col_idx must be ascending per row;
 * chunk a positive multiple of 32; lanes_per_row 8, 16 or 32.  Errors: INVALID_ARG,
 * BAD_CSR (row_ptr not monotone from 0, or a row not ascending). */
ion_status ion_csr_bank_order(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t chunk,
                              int32_t lanes_per_row, int32_t *perm);

/* Test hook, never called in production: the device allocation that follows the next
 * `after` ones (in any handle of the process) reports out-of-memory, once, so that the
 * error paths of creation and setup can be exercised; a negative value disarms it. */
ion_status ion_debug_fail_alloc(int32_t after);

/* Steps taken so far (the absolute index of the next step). */
int64_t ion_step_count(const ion_sim *sim);

/* Set the absolute index of the next step (checkpoint resume: write the saved state,
 * then set the saved step count so evoked-input pulses line up).  Synchronises. */
ion_status ion_set_step_count(ion_sim *sim, int64_t t);

/* Number of kernel launches the handle issued (graph nodes counted once per replay). */
int64_t ion_launch_count(const ion_sim *sim);

/* Human-readable description of the last error on this handle (NULL: the last error of
 * a call that had no handle yet, e.g. a failed ion_create). */
const char *ion_last_error(const ion_sim *sim);

void ion_destroy(ion_sim *sim);

/* ---- single-launch primitives (one step of one stage; device pointers) ------------ */

/* Ic[i] = g_c * sum_j (0.8 e^{-(V_i-V_j)^2/100} + 0.2)(V_i - V_j) for a dense uniform
 * network (Algorithm 1 with C = 100 %).  vdend, ic: device arrays of n floats.
 * kahan != 0 compensates the j sums.  The launch stages V_dend into shared memory with
 * bulk copies whose completion it waits for with a bound (about 0.5 s); should a copy not
 * land in time, the rows of the affected thread blocks receive NaN instead of a current
 * (this entry point has no status word to report it otherwise). */
ion_status ion_gj_dense(const float *vdend, int32_t n, float g_c, float *ic, int32_t kahan,
                        void *cuda_stream);

/* Same currents as ion_gj_dense, computed without allocating any memory.
 *
 * The paper has no counterpart of this entry point.  It exists for callers that must not
 * allocate: a simulation loop with a hard per-step deadline (an allocation can block or
 * synchronise the device), code running while a stream is being captured into a CUDA
 * graph, and host programs whose device memory belongs to their own allocator.
 * ion_gj_dense takes its scratch (V_dend copied and padded to a multiple of 256 floats)
 * from the stream-ordered allocator; this variant keeps that scratch in a fixed device
 * array compiled into the library, 65536 floats (256 KiB) on every GPU that loads it,
 * held until the process exits.  So n rounded up to a multiple of 256 may be at most
 * 65536; a larger n returns ION_ERR_INVALID_ARG without touching the device.
 * Arguments, layout and result are those of ion_gj_dense.
 * The first call on each device looks up the array's device address with that device
 * current: make that first call before starting any stream capture.  The address is kept
 * with the identity of the device's context; after a device reset (which gives the device
 * a new context and reloads the library's device code) the next call looks it up again,
 * so that call too belongs outside a capture.
 * Every call on a device shares the one array and leaves its contents behind; each call
 * rewrites the whole range it reads, so nothing needs clearing between calls.  Calls
 * whose work can overlap on the GPU (other streams, other host threads) race on the
 * array: the caller must order them. */
ion_status ion_gj_dense_noalloc(const float *vdend, int32_t n, float g_c, float *ic, int32_t kahan,
                                void *cuda_stream);

/* Ic[i] = sum_{e in row i} w[e] (0.8 e^{-dV^2/100} + 0.2) dV, dV = V_i - V_{col[e]}
 * (Algorithm 1 over a CSR matrix).  All arrays on the device; w NULL means every
 * weight is g_c. */
ion_status ion_gj_csr(const float *vdend, int32_t n, const int32_t *row_ptr,
                      const int32_t *col_idx, const float *w, float g_c, float *ic,
                      void *cuda_stream);

/* One explicit-Euler cell update of n cells, in place on the device SoA buffer
 * state[19 * n] (V_dend included), with gap current ic[n] (NULL: none) and evoked
 * current iapp[n] (NULL: none).  model NULL = default. */
ion_status ion_cell_update(float *state, int32_t n, const float *ic, const float *iapp,
                           const ion_model *model, double dt_ms, void *cuda_stream);

/* ---- measurement ------------------------------------------------------------------ */

/* Throughput probe of one execution unit at the current clock: what = 0 measures SFU
 * ex2.approx results per second, what = 1 FP32 FMAs per second, what = 2 tanh.approx.bf16x2
 * instructions per second (two activations each), over the whole GPU
 * (8 independent chains per thread, 8 CTAs of 256 threads per SM, `iters` rounds).
 * These are the measured denominators of the dense gap-junction kernel's roofline.
 * Synchronises the stream.  Not part of the paper's method. */
ion_status ion_probe_peak(int32_t what, int32_t iters, void *cuda_stream, double *rate_out);

/* ---- learned surrogate of the rate functions ------------------------------------ */
/* Not in the paper.  An MLP (V, [Ca]) -> 64 tanh -> 64 tanh -> 24 outputs stands in for
 * the gates' rate functions when ION_FLAG_SURROGATE is set (ion_params.surrogate points
 * at an ion_surrogate_weights): output 2g is logit(x_inf) of gate g, clipped to +-15 (gate
 * order r s q k l m_s h_s n_s x_s m_a h_a x_a), output 2g+1 is ln(tau_g) (unused for
 * m_s, m_a).  Inputs are
 * x = ((V - in_shift[0]) in_scale[0], (ln [Ca] - in_shift[1]) in_scale[1]); outputs are
 * y = y' out_scale + out_shift.  Weights row-major [out][in], FP32; inference converts
 * the 64x64 and 64x24 layers to BF16 and runs them on the tensor cores (FP32
 * accumulation), fused with the cell update. */
#define ION_MLP_IN 2
#define ION_MLP_HID 64
#define ION_MLP_OUT 24
typedef struct {
    float w1[ION_MLP_HID * ION_MLP_IN], b1[ION_MLP_HID];
    float w2[ION_MLP_HID * ION_MLP_HID], b2[ION_MLP_HID];
    float w3[ION_MLP_OUT * ION_MLP_HID], b3[ION_MLP_OUT];
    float in_shift[ION_MLP_IN], in_scale[ION_MLP_IN];
    float out_shift[ION_MLP_OUT], out_scale[ION_MLP_OUT];
} ion_surrogate_weights;

typedef struct {
    int64_t n_samples;   /* training set size (e.g. 1e6), >= 256                    */
    int32_t epochs;      /* passes over the set (each with its own reshuffle)       */
    int32_t batch;       /* minibatch size, a multiple of 128, <= n_samples          */
    float lr;            /* Adam step size (cosine-decayed to 1 % over the run)     */
    uint64_t seed;       /* samples and initial weights                             */
    float v_lo, v_hi;    /* V range, mV (uniform)                                   */
    float ca_lo, ca_hi;  /* [Ca] range (log-uniform), > 0                           */
    void *cuda_stream;
} ion_train_cfg;

/* Train the surrogate on the GPU: draw n_samples (V, [Ca]) on the device, label them with
 * the exact FP32 rate functions, normalise (per-output mean / standard deviation), fit
 * by minibatch Adam with the library's own forward / backward kernels (FP32, partial
 * gradients summed in a fixed order).  weights_out: host struct, filled on success;
 * final_loss (nullable): mean masked squared error of the last epoch, normalised units.
 * Synchronises the stream. */
ion_status ion_surrogate_train(const ion_train_cfg *cfg, ion_surrogate_weights *weights_out,
                               float *final_loss);

/* Gradient of the training loss L = sum_{s,o} mask_o (y_so - t_so)^2 / (B sum(mask)) for
 * one batch, computed by the training kernels: x (B x 2, normalised inputs), t (B x 24,
 * normalised targets), mask (24) are host arrays; grad receives dL/dparams in the
 * weights' layout (w1..b3; the normalisation fields are left untouched); loss
 * (nullable) receives L.  Synchronises. */
ion_status ion_surrogate_grad(const ion_surrogate_weights *weights, const float *x, const float *t,
                              const float *mask, int32_t B, ion_surrogate_weights *grad, float *loss);

/* Evaluate the surrogate on the tensor cores (BF16 weights and activations, FP32
 * accumulation) for n host pairs (V[i], ca[i]); out (host, n x 24) in physical units. */
ion_status ion_surrogate_eval(const ion_surrogate_weights *weights, const float *V, const float *ca,
                              int64_t n, float *out);

#ifdef __cplusplus
}
#endif
#endif /* ION_H */
