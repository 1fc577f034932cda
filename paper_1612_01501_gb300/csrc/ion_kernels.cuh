// ion_kernels.cuh -- launch arguments and launchers shared by the library's .cu files.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "ion.h"
#include "ion_async.cuh"
#include "ion_model.cuh"

namespace ion {

// Dense tiles of V_dend are staged TJ floats at a time; every V_dend buffer is padded
// to a multiple of PAD_J floats with a sentinel voltage far from any physiological
// value, so padded pairs contribute exactly 0 to the exponential sum.
constexpr int TJ = 8192;
constexpr int CSR_CHUNK = 32768;   // floats of V_dend per shared-memory chunk (128 KB)
static_assert(CSR_CHUNK <= 65536, "16-bit chunk-relative columns need chunks of at most 2^16 cells");
constexpr int PAD_J = 256;
constexpr float PAD_VOLT = 1.0e7f;

// Scale s with (s dV)^2 = dV^2 log2(e) / 100, so e^{-dV^2/100} = 2^{-(s dV)^2}.
constexpr float GJ_SCALE = 0.12011224087864498f;   // sqrt(log2(e) / 100)

struct StepCommon {
    StateView S;          // 20 * stride floats: fields 0..18 and the second V_dend slot
    int32_t n;            // cells
    int32_t n_pad;        // V_dend length incl. sentinel padding (multiple of PAD_J)
    const int64_t *t_dev; // absolute index of the first step of the current replay (NULL: t = 0)
    int32_t k_off;        // this launch's step offset from *t_dev
    int32_t par;          // parity of this launch's step index t (the V_dend slot of step t),
                          // passed by the host so that the slot address does not wait on *t_dev;
                          // -1 in persistent launches (which run many steps)
    int32_t vd_fixed;     // 1: V_dend is updated in place in slot 0 (single-cell-launch primitives)
    PulseTable pulses;
    const float *iapp;    // dense evoked input of this step (n floats) or NULL
    uint32_t *status;     // sticky status word
    float *trace;         // V_axon ring [cap][n] or NULL
    int32_t trace_stride, trace_cap;
    int32_t pdl;          // host side: launch with programmatic stream serialization
    ModelF P;
};

// Launch a per-step kernel; with `pdl`, with programmatic stream serialization, so that
// its CTAs may be scheduled while the kernel before it drains (the kernel starts with
// pdl_enter(), which waits for that kernel's completion before any global access).
template <class... P, class... A>
inline cudaError_t launch_k(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                            A... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// V_dend slot holding step t: slot 0 is field F_VDEND, slot 1 is field 19.
__device__ __forceinline__ float *vd_slot(const StateView &S, int64_t t) {
    return S.base + ((t & 1) ? 19 : 0) * S.stride;
}
__device__ __forceinline__ int64_t step_index(const StepCommon &c) {
    return c.t_dev != nullptr ? *c.t_dev + c.k_off : (int64_t)c.k_off;
}
__device__ __forceinline__ float *vd_cur(const StepCommon &c) {
    return c.vd_fixed ? c.S.base : vd_slot(c.S, c.par);
}
__device__ __forceinline__ float *vd_next(const StepCommon &c) {
    return c.vd_fixed ? c.S.base : vd_slot(c.S, c.par + 1);
}

// Write the step result of cell i (and its trace sample, status bit).
__device__ __forceinline__ void finish_cell(const StepCommon &a, int64_t t, float *vd_next, int64_t i,
                                            const CellNext &o) {
    store_cell(a.S, vd_next, i, o);
    if (!cell_finite(o)) atomicOr(a.status, (uint32_t)ST_NONFINITE);
    if (a.par >= 0 && (int)(t & 1) != a.par) atomicOr(a.status, (uint32_t)ST_SLOT);   // host and device disagree
    if (a.trace != nullptr && ((t + 1) % a.trace_stride) == 0) {
        const int64_t sample = (t + 1) / a.trace_stride - 1;
        a.trace[(sample % a.trace_cap) * (int64_t)a.n + i] = o.va;
    }
}

// ---- split cell update ------------------------------------------------------------------
// The explicit-Euler update of one cell is a chain of ~36 SFU and ~300 FP32 operations when
// one thread does it.  A CTA whose rows are few next to its threads (the dense step) spreads
// each cell's outputs over NROLE threads instead: role 0 the dendrite (V_dend, [Ca], I_CaH,
// I_c, s), 1 the soma voltage (and m_s), 2 the axon voltage (m_a, the trace sample), 3..9
// the remaining gates.  Every role calls the same functions as cell_step, so a cell gets
// the same bits either way.
constexpr int NROLE = 10;
constexpr int NCW = 15;   // words of Cell
// state field of Cell word w (word 0, V_dend, comes from the step's V_dend slot)
__device__ __forceinline__ int cell_word_field(int w) {
    return w == 0 ? -1 : (w <= 8 ? w : (w <= 11 ? w + 1 : w + 2));
}

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Start copying the 15 Cell words of rows [row_base, row_base + rows) into cs[w * rows + r]
// (all threads; waited for with cp_async_wait_all).  Rows at or past n are skipped.
__device__ __forceinline__ void stage_cells(float *cs, const StateView &S, const float *vcur, int64_t row_base,
                                            int rows, int n) {
    for (int q = threadIdx.x; q < NCW * rows; q += blockDim.x) {
        const int w = q / rows, r = q - w * rows;
        const int64_t i = row_base + r;
        if (i >= n) continue;
        const float *src = w == 0 ? vcur : S.f(cell_word_field(w));
        cp_async4(cs + q, src + i);
    }
    cp_async_commit();
}

__device__ __forceinline__ Cell staged_cell(const float *cs, int rows, int r) {
    Cell c;
    c.vd = cs[0 * rows + r];
    c.vs = cs[1 * rows + r];
    c.va = cs[2 * rows + r];
    c.ca = cs[3 * rows + r];
    c.r = cs[4 * rows + r];
    c.s = cs[5 * rows + r];
    c.q = cs[6 * rows + r];
    c.k = cs[7 * rows + r];
    c.l = cs[8 * rows + r];
    c.hs = cs[9 * rows + r];
    c.ns = cs[10 * rows + r];
    c.xs = cs[11 * rows + r];
    c.ha = cs[12 * rows + r];
    c.xa = cs[13 * rows + r];
    c.gcal = cs[14 * rows + r];
    return c;
}

// Where a role writes the step-(t+1) words of cell i: the global state (per-step kernels)
struct RoleOutGlobal {
    StateView S;
    __device__ __forceinline__ void put(int field, int64_t i, int, float v) const { S.f(field)[i] = v; }
    __device__ __forceinline__ void put_vd(int, float) const {}   // V_dend goes to the next slot only
};
// ... or a CTA's shared-memory copy of its rows' state (persistent kernels): the 15 Cell
// words in cs[w * rows + r] (word order of Cell) and the four output-only words (m_s, m_a,
// I_CaH, I_c) in xs[k * rows + r]
struct RoleOutSmem {
    float *cs, *xs;
    int rows;
    __device__ __forceinline__ float *slot(int field) const {
        switch (field) {
            case F_MS: return xs;
            case F_MA: return xs + rows;
            case F_ICAH: return xs + 2 * rows;
            case F_IC: return xs + 3 * rows;
            default: return cs + (field <= F_L ? field : (field <= F_XS ? field - 1 : field - 2)) * rows;
        }
    }
    __device__ __forceinline__ void put(int field, int64_t, int r, float v) const { slot(field)[r] = v; }
    __device__ __forceinline__ void put_vd(int r, float v) const { cs[r] = v; }
};

// Outputs of one role of cell i (local row r of its CTA; see NROLE); iapp is read by role 0
// only.  V_dend(t+1) always goes to the global next slot (other CTAs read it).
template <class Out>
__device__ __forceinline__ void cell_step_role(int role, const StepCommon &a, int64_t t, float *vd_next, int64_t i,
                                               int r, const Cell &c, float ic, float iapp, const Out &out) {
    const ModelF &P = a.P;
    const float dt = P.dt;
    switch (role) {
        case 0: {
            const DendNext d = dend_step(P, c, ic, iapp);
            vd_next[i] = d.vd;
            out.put_vd(r, d.vd);
            out.put(F_CA, i, r, d.ca);
            out.put(F_ICAH, i, r, d.icah);
            out.put(F_IC, i, r, ic);
            out.put(F_S, i, r, relax(c.s, rate_s(c.ca), dt));
            if (!(isfinite(d.vd) && isfinite(d.ca))) atomicOr(a.status, (uint32_t)ST_NONFINITE);
            if (a.par >= 0 && (int)(t & 1) != a.par) atomicOr(a.status, (uint32_t)ST_SLOT);
            break;
        }
        case 1: {
            const float ms = minf_na(c.vs);
            const float vs = soma_step(P, c, ms);
            out.put(F_VSOMA, i, r, vs);
            out.put(F_MS, i, r, ms);
            if (!isfinite(vs)) atomicOr(a.status, (uint32_t)ST_NONFINITE);
            break;
        }
        case 2: {
            const float ma = minf_na(c.va);
            const float va = axon_step(P, c, ma);
            out.put(F_VAXON, i, r, va);
            out.put(F_MA, i, r, ma);
            if (!isfinite(va)) atomicOr(a.status, (uint32_t)ST_NONFINITE);
            if (a.trace != nullptr && ((t + 1) % a.trace_stride) == 0) {
                const int64_t sample = (t + 1) / a.trace_stride - 1;
                a.trace[(sample % a.trace_cap) * (int64_t)a.n + i] = va;
            }
            break;
        }
        case 3: out.put(F_R, i, r, relax(c.r, rate_r(c.vd), dt)); break;
        case 4: out.put(F_Q, i, r, relax(c.q, rate_q(c.vd), dt)); break;
        case 5:
            out.put(F_K, i, r, relax(c.k, rate_k(c.vs), dt));
            out.put(F_HS, i, r, relax(c.hs, rate_hs(c.vs), dt));
            break;
        case 6: out.put(F_L, i, r, relax(c.l, rate_l(c.vs), dt)); break;
        case 7:
            out.put(F_NS, i, r, relax(c.ns, rate_ns(c.vs), dt));
            out.put(F_HA, i, r, relax(c.ha, rate_ha(c.va), dt));
            break;
        case 8: out.put(F_XS, i, r, relax(c.xs, rate_x(c.vs), dt)); break;
        default: out.put(F_XA, i, r, relax(c.xa, rate_x(c.va), dt)); break;
    }
}

// All 18 words of a single-thread step into the shared-memory copy (persistent kernels).
__device__ __forceinline__ void put_cell_smem(const RoleOutSmem &out, int r, const CellNext &o) {
    out.put_vd(r, o.vd);
    out.put(F_VSOMA, 0, r, o.vs);
    out.put(F_VAXON, 0, r, o.va);
    out.put(F_CA, 0, r, o.ca);
    out.put(F_R, 0, r, o.r);
    out.put(F_S, 0, r, o.s);
    out.put(F_Q, 0, r, o.q);
    out.put(F_K, 0, r, o.k);
    out.put(F_L, 0, r, o.l);
    out.put(F_MS, 0, r, o.ms);
    out.put(F_HS, 0, r, o.hs);
    out.put(F_NS, 0, r, o.ns);
    out.put(F_XS, 0, r, o.xs);
    out.put(F_MA, 0, r, o.ma);
    out.put(F_HA, 0, r, o.ha);
    out.put(F_XA, 0, r, o.xa);
    out.put(F_ICAH, 0, r, o.icah);
    out.put(F_IC, 0, r, o.ic);
}

struct DenseArgs {
    StepCommon c;
    float g;              // uniform pair weight
    int32_t fuse;         // 1: cell update in the same launch; 0: write Ic only
    int32_t kahan;
    float *ic_out;        // when !fuse: Ic[n]
    const float *vd_in;   // when !fuse: V_dend[n_pad] (sentinel padded)
};
struct CsrArgs {
    StepCommon c;
    const int32_t *row_ptr;
    const int32_t *col;
    const uint16_t *col16;   // non-NULL: the low 16 bits of every column (see ion_csr.cu)
    const float *w;       // NULL: every weight is g
    float g;
    int32_t fuse;
    float *ic_out;
    const float *vd_in;
    int32_t lin;          // 1: linear junctions (SGJ use case); needs col16
    // staged kernel, padded layout (see ion_sim): columns, weights, segment offsets
    const uint16_t *col16p;
    const float *wp;
    const int32_t *segoff;
};
struct PersistArgs {
    StepCommon c;         // k_off unused: the launch runs steps *t_dev .. *t_dev + n_steps - 1
    float g;
    int32_t n_steps;
    int32_t kahan;
    uint32_t *bar_count;  // grid-barrier arrivals (set to bar_base before the launch)
    uint32_t *abort_flag; // set by a CTA whose wait timed out (zeroed before the launch)
    uint32_t *bar_flag;   // the last arrival's release flag (set to bar_base before the launch)
    uint64_t timeout_ns;  // bound on one grid-barrier wait
    int64_t debug_delay_ns;  // test hook: the last CTA sleeps this long before its first step
    uint32_t bar_base;    // the arrival counter's value at launch (0; a test hook sets others)
};
struct HalfArgs {
    StepCommon c;          // k_off unused: the launch runs steps *t_dev .. *t_dev + n_steps - 1
    float g;
    int32_t n_steps;
    int32_t rows;          // rows per CTA (the block size b)
    uint32_t *bar_count;   // grid-barrier arrivals (set to bar_base before the launch)
    uint32_t *abort_flag;
    uint64_t timeout_ns;
    int64_t debug_delay_ns;
    uint32_t bar_base;     // the arrival counter's value at launch
    float *colsum;         // [grid][colsum_stride] column sums of each CTA's tile (L2-resident)
    int32_t colsum_stride;
    float *usum;           // [grid] sum of u over each CTA's own rows
    int32_t chunk;         // tile columns per column-partial round (a multiple of 128; set by the launcher)
};
struct MatrixArgs {
    StepCommon c;
    const float *W;       // n rows x n_pad columns, row-major, zero beyond column n
};
struct CellArgs {
    StepCommon c;
    const float *ic;      // NULL: no gap current
    const float *cellp;   // NULL, or per-cell constants: NCELLP x c.S.stride floats, row k
                          // holding member k of ModelF (g_ds ... VL) for every cell
};

// launchers (return the CUDA launch status)
cudaError_t launch_dense_step(const DenseArgs &a, int rows_per_warp, int warps, int col_splits, cudaStream_t st);
cudaError_t launch_csr_step(const CsrArgs &a, int lanes_per_row, int rows_per_cta, cudaStream_t st);
cudaError_t prepare_csr_step();
cudaError_t launch_csr_chunk_step(const CsrArgs &a, int lanes_per_row, int rows_per_cta, const int32_t *mid,
                                  int n_chunks, bool prepare, cudaStream_t st);
cudaError_t prepare_matrix_step(int n_pad);
cudaError_t launch_matrix_step(const MatrixArgs &a, int R, cudaStream_t st);   // R: rows per warp, 1, 2 or 4
int matrix_default_R(int n, int sms);
int sgj_partials(int n);   // CTAs of the SGJ partial-sum launch (the update reads that many)
constexpr int SGJ_ONE_LAUNCH = 16384;   // SGJ dense networks up to this size take one launch per step
cudaError_t launch_sgj_dense_step(const StepCommon &c, float g, float *part, cudaStream_t st);
cudaError_t launch_sgj_csr_step(const CsrArgs &a, cudaStream_t st);
cudaError_t launch_csr_col16(const int32_t *col, int64_t nnz, int64_t n_alloc, uint16_t *col16, cudaStream_t st);
cudaError_t launch_csr_half_step(const CsrArgs &a, int lanes_per_row, int rows_per_cta, const int32_t *split,
                                 const int32_t *rev, float *slot, float *icu, cudaStream_t st);
cudaError_t launch_csr_pad_fill(const int32_t *row_ptr, const int32_t *mid, const int32_t *col, const float *w,
                                 int32_t n, int n_chunks, int rows, int nb, const int32_t *off, uint16_t *col16p,
                                 float *wp, cudaStream_t st);
cudaError_t launch_csr_chunk_bounds(const int32_t *row_ptr, const int32_t *col, int32_t n, int n_chunks,
                                    int32_t *mid, cudaStream_t st);
size_t csr_chunk_smem_bytes(int n_pad, int rows);
cudaError_t launch_cell_step(const CellArgs &a, cudaStream_t st);
cudaError_t launch_advance(int64_t *t_dev, int64_t k, cudaStream_t st);
cudaError_t launch_fill(float *p, float v, int64_t n, cudaStream_t st);
cudaError_t launch_rates(float V, float ca, float *xinf_tau /*24 floats, device*/, cudaStream_t st);
cudaError_t launch_default_state(const ModelF &P, float V0, float ca0, float gcal, int32_t n, int64_t stride,
                                 float *state, cudaStream_t st);
cudaError_t prepare_dense_step(int rows_per_warp, int warps, int col_splits, int n_pad);
cudaError_t persist_dense(const PersistArgs &a, int rows_per_warp, int warps, int col_splits, int *grid_out,
                          bool launch, cudaStream_t st);
cudaError_t launch_dense_half(const HalfArgs &a, int rows_per_warp, int warps, int col_splits, int grid,
                              bool launch, int *ok_out, cudaStream_t st);
int half_colsum_stride(int grid, int rows_per_cta);
int dense_max_threads(int rows_per_warp);     // thread limit of the step kernel
int persist_max_threads(int rows_per_warp);   // thread limit of the persistent kernel

// shared-memory size of a dense launch
size_t dense_smem_bytes(int n_pad, int rows_per_warp, int warps);

// surrogate inference on tcgen05 (ion_mlp_tc.cu): packed weights, cell kernel, batched eval
size_t surrogate_tc_weights_bytes();
cudaError_t surrogate_tc_prepare();
cudaError_t surrogate_tc_pack(const ion_surrogate_weights *d_w, void *d_out, cudaStream_t st);
cudaError_t launch_surrogate_tc(const StepCommon &c, const void *W, const float *ic, cudaStream_t st);
cudaError_t launch_mlp_eval_tc(const void *W, int64_t n, const float *V, const float *ca, float *out,
                               uint32_t *status, cudaStream_t st);

}  // namespace ion
