// ion_sim.h -- the handle behind the opaque `ion_sim` of include/ion.h (library-internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ion.h"
#include "ion_kernels.cuh"

struct ion_sim {
    // network (batches: n = padded total, n_user = cells in the user's numbering, and
    // d_map[user cell] = padded cell)
    int32_t n = 0, kind = 0, n_pad = 0;
    int64_t n_user = 0;
    int32_t *d_map = nullptr;
    int64_t stride = 0;
    float g = 0.0f;                 // dense pair weight / CSR default weight
    int64_t nnz = 0;
    int32_t *d_rowptr = nullptr, *d_col = nullptr;
    float *d_w = nullptr;
    bool own_csr = false;
    uint16_t *d_col16 = nullptr;    // low 16 bits of every column (compact CSR layout)
    float *d_sgj = nullptr;         // SGJ dense: per-CTA partial sums of V_dend - m
    float *d_W = nullptr;           // dense matrix: n rows x n_pad columns (zero padded)
    // state and bookkeeping
    float *d_state = nullptr;       // 20 * stride floats
    float *d_ic = nullptr;          // gap currents (split mode)
    float *d_cellp = nullptr;       // per-cell constants, NCELLP rows of stride floats (or NULL)
    int64_t *d_t = nullptr;         // device step counter
    uint32_t *d_status = nullptr;   // sticky status bits
    uint32_t sticky = 0;            // status bits seen by the host
    int64_t t = 0;                  // host step counter (steps enqueued)
    int64_t launches = 0;           // kernel launches issued (graph nodes counted per replay)
    // evoked input
    int32_t *d_poff = nullptr;
    int64_t *d_pbeg = nullptr, *d_pend = nullptr;
    float *d_pamp = nullptr;
    int32_t n_pulses = 0;
    float *d_iapp = nullptr;
    int64_t iapp_cap = 0;
    // trace
    float *d_trace = nullptr;
    int32_t trace_stride = 0, trace_cap = 0;
    int64_t trace_read = 0;
    // asynchronous trace drain: copy stream, events, and the first sample index whose slot
    // a pending copy still reads (steps producing it wait for the copy)
    cudaStream_t copy_st = nullptr;
    cudaEvent_t ev_ready = nullptr, ev_copied = nullptr;
    bool copy_pending = false;
    int64_t copy_guard_sample = 0;
    // model and launch configuration
    ion_model model{};
    ion::ModelF P{};
    double dt = 0.05;
    cudaStream_t st = nullptr;
    cudaStream_t own_stream = nullptr;   // created when the caller passed no stream
    uint32_t flags = 0;
    int32_t graph_steps = 50, check_every = 64;
    uint64_t barrier_timeout_ns = 0;
    int64_t debug_delay_ns = 0;
    uint32_t *d_bar = nullptr;      // grid barrier counter + abort word (persistent launches)
    uint32_t barrier_base = 0;      // the counter's value at each persistent launch (test hook)
    uint32_t bar_init[64] = {};     // host source of the barrier reset (lives with the handle)
    int persist_R = 0, persist_W = 0, persist_GJ = 1;
    float *d_half = nullptr;        // half-work persistent kernel: column sums + per-CTA sums of u
    int half_grid = 0, half_stride = 0;
    int device = 0, sms = 1;
    int dense_R = 1, dense_W = 4, dense_GJ = 1, csr_SW = 8, csr_rows = 256;
    int csr_staged = 0;             // 1: V_dend staged in shared memory chunk by chunk
    int csr_chunk_SW = 32, csr_chunk_rows = 0, n_chunks = 1;
    int32_t *d_mid = nullptr;       // interior chunk boundaries per row
    // the staged kernel's padded layout: each (chunk, row) segment's columns chunk-relative
    // and padded to whole 16-byte groups with entries that index the row's own V_dend
    // (a pair with dV = 0 adds exactly 0); segments in chunk-major order from d_segoff
    uint16_t *d_col16p = nullptr;
    float *d_wp = nullptr;
    int32_t *d_segoff = nullptr;
    int32_t pad_rows = 0;           // rows per CTA the padding entries are numbered for
    bool col16_bank = false;        // col16 holds the opt-in bank order (no padded layout)
    // half-work CSR (ION_FLAG_HALF_WORK on a CSR network): first upper edge of each row, the
    // mirrored position of every upper edge, the per-edge slots, the rows' upper sums
    int32_t *d_split = nullptr, *d_rev = nullptr;
    float *d_slot = nullptr, *d_icu = nullptr;
    void *d_mlp = nullptr;          // packed surrogate weights (ION_FLAG_SURROGATE), warp-MMA layout
    void *d_mlp_tc = nullptr;       // the same weights in the tcgen05 kernels' layout
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};   // K-step graphs, by the parity of their first step
    int64_t t_enq = 0;              // the device step counter's value where the next launch is enqueued
    int64_t graph_launches = 0;
    bool no_graph = false;
    bool pdl_off = false;   // programmatic launches unavailable (graph capture refused them)
    std::string err;

    // extension points (persistent, batched and surrogate variants)
    cudaError_t (*step_override)(ion_sim *, int k_off, const float *iapp) = nullptr;
    ion_status (*run_override)(ion_sim *, int64_t n_steps, const float *iapp) = nullptr;
    ion_status (*prepare_hook)(ion_sim *) = nullptr;
    ion_status (*state_sync_hook)(ion_sim *) = nullptr;
    ion_status (*state_load_hook)(ion_sim *) = nullptr;
    void (*extra_free)(ion_sim *) = [](ion_sim *) {};
    void (*drop_hook)(ion_sim *) = nullptr;   // drops graphs an extension captured
    void *ext = nullptr;            // extension state
    int64_t lps = 1;                // kernel launches per step

    int64_t launches_per_step() const { return lps; }
};

// Device allocation of every handle buffer; a test hook (ion_debug_fail_alloc) can make one
// call report out-of-memory so that the error paths are exercised without a real shortage.
cudaError_t ion_dev_alloc(void **p, size_t bytes);
template <class T>
inline cudaError_t ion_alloc(T **p, size_t bytes) {
    return ion_dev_alloc(reinterpret_cast<void **>(p), bytes);
}

// shared helpers (ion_api.cu)
void ion_csr_fill(const ion_sim *s, ion::CsrArgs &a, bool staged);
ion_status ion_prepare_csr_chunk(ion_sim *s);
ion_status ion_fail(ion_sim *s, ion_status code, const char *fmt, ...);
ion::ModelF ion_model_to_f32(const ion_model &m, double dt);
ion_status ion_cell_params_to_f32(const float *cp, int32_t n, const ion_model &m, double dt, std::vector<float> &out);
ion::StepCommon ion_step_common(ion_sim *s, int k_off, const float *iapp);
float *ion_field_ptr(ion_sim *s, int32_t field);
ion_status ion_validate_csr(int32_t n, const ion_conn *c);
void ion_choose_dense_shape(int n, int sms, int *R, int *W, int *GJ);
void ion_choose_csr_shape(double mean_deg, int *SW, int *rows);
// 16-bit columns of a sorted host CSR in shared-memory bank order (ion_bank.cu)
bool ion_csr_bank_col16(int32_t n, int32_t n_pad, const int32_t *row_ptr, const int32_t *col,
                        std::vector<uint16_t> &out);
ion_status ion_setup_csr_staging(ion_sim *s, int mode);
ion_status ion_setup_csr_half(ion_sim *s, const ion_conn *conn);
void ion_sim_free_device(ion_sim *s);
// destroy the captured step graphs (after any change they depend on)
inline void ion_drop_graphs(ion_sim *s) {
    for (cudaGraphExec_t &g : s->gexec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    if (s->drop_hook) s->drop_hook(s);
}
// per-flag setup of the extensions (ion_ext.cu)
ion_status ion_sim_setup_extras(ion_sim *s, const ion_params *p);
// batch state I/O in the user's numbering (ion_batch.cu)
ion_status ion_batch_read(ion_sim *s, int32_t field, float *out);
ion_status ion_batch_write(ion_sim *s, int32_t field, const float *in);
int32_t ion_batch_map_cell(ion_sim *s, int64_t user_cell);
// surrogate (ion_mlp.cu)
ion_status ion_setup_surrogate(ion_sim *s, const ion_params *p);
