// ion_csr.cu -- sparse (CSR) gap-junction step and the stand-alone cell update.
//
// Algorithm 1 over a programmed weight matrix (Sec. 2.3): for every stored connection
// e = (i, j) of row i,
//   Ic_i += w_e (0.8 e^{-dV^2/100} + 0.2) dV,  dV = V_dend,i - V_dend,j.
// A CTA of 256 threads owns `rows` consecutive rows (1..256, chosen from the mean degree
// so that the grid keeps every SM busy).  Phase 1: groups of SW lanes (SW = 1..32) walk
// one row's edges; with 16-byte aligned arrays each lane reads four consecutive indices
// and weights per 16-byte load, and four V_dend gathers are in flight per lane; the SW
// lane sums are combined with shuffles in a fixed order.  Phase 2: one thread per row
// runs the explicit-Euler cell update with that row's current (fused variant), so the
// cell work runs on full warps whatever SW is.
#include <cuda_runtime.h>

#include <algorithm>

#include "ion_async.cuh"
#include "ion_csr_core.cuh"
#include "ion_kernels.cuh"

namespace ion {

// One CTA of 256 threads owns `rows` consecutive rows (rows <= 256).  Phase 1: groups of
// SW lanes take the rows round-robin; phase 2: thread t updates row t.  LIN: linear
// junctions (the SGJ use case), on the 16-bit column layout only.
template <int SW, bool VEC, bool HAS_W, bool C16, bool LIN = false>
__global__ void __launch_bounds__(256) csr_step_kernel(const CsrArgs a, int rows) {
    static_assert(!LIN || C16, "linear junctions run on the 16-bit column layout");
    __shared__ float ic_s[256];
    pdl_enter();
    const StepCommon &c = a.c;
    const int n = c.n;
    const int row0 = blockIdx.x * rows;
    const int64_t t = step_index(c);
    const float *vcur = a.vd_in != nullptr ? a.vd_in : vd_cur(c);
    float *vnext = a.fuse ? vd_next(c) : nullptr;
    const int sub = threadIdx.x / SW, li = threadIdx.x % SW, nsub = blockDim.x / SW;
    const int iters = (rows + nsub - 1) / nsub;          // the same for every lane (shuffles below)
    // a row's bounds and V_dend are loaded one row ahead (see the chunked variant)
    auto bounds = [&](int it, int &e0, int &e1, float &vi) {
        const int rr = sub + it * nsub, i = row0 + rr;
        e0 = e1 = 0;
        vi = 0.0f;
        if (it < iters && rr < rows && i < n) {
            e0 = a.row_ptr[i];
            e1 = a.row_ptr[i + 1];
            vi = vcur[i];
        }
    };
    int e0n, e1n;
    float vin;
    bounds(0, e0n, e1n, vin);
    for (int it = 0; it < iters; ++it) {
        const int rr = sub + it * nsub;
        const int e0 = e0n, e1 = e1n;
        const float vi = vin;
        bounds(it + 1, e0n, e1n, vin);
        float acc = 0.0f;
        if (e1 > e0) {   // rows past the end (and empty rows) have e0 == e1
            if (C16)
                acc = csr_row_sum16<SW, HAS_W, false, LIN>(a.col16, a.w, e0, e1, vi, li, VjGlobal{vcur});
            else
                acc = csr_row_sum<SW, VEC, HAS_W>(vcur, a.col, a.w, e0, e1, vi, li);
        }
#pragma unroll
        for (int off = SW / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (li == 0 && rr < rows) ic_s[rr] = (HAS_W ? acc : acc * a.g) * (1.0f / GJ_SCALE);
    }
    __syncthreads();
    if ((int)threadIdx.x >= rows) return;
    const int i = row0 + threadIdx.x;
    if (i >= n) return;
    const float ic = ic_s[threadIdx.x];
    if (!a.fuse) {
        a.ic_out[i] = ic;
        return;
    }
    const Cell cell = load_cell(c.S, vcur, i);
    float iapp = pulse_current(c.pulses, i, t);
    if (c.iapp != nullptr) iapp += c.iapp[i];
    const CellNext o = cell_step(c.P, cell, ic, iapp);
    finish_cell(c, t, vnext, i, o);
}

template <int SW, bool VEC, bool HAS_W, bool C16 = false, bool LIN = false>
static cudaError_t launch_csr_T(const CsrArgs &a, int rows, cudaStream_t st) {
    const int grid = (a.c.n + rows - 1) / rows;
    return launch_k(csr_step_kernel<SW, VEC, HAS_W, C16, LIN>, dim3(grid), dim3(256), 0, st, a.c.pdl != 0, a, rows);
}
template <int SW>
static cudaError_t launch_csr_SW(const CsrArgs &a, int rows, cudaStream_t st) {
    if (a.lin) {
        if (a.col16 == nullptr) return cudaErrorInvalidValue;
        return a.w != nullptr ? launch_csr_T<SW, true, true, true, true>(a, rows, st)
                              : launch_csr_T<SW, true, false, true, true>(a, rows, st);
    }
    if (a.col16 != nullptr)   // 16-byte aligned indices (and weights, checked at creation)
        return a.w != nullptr ? launch_csr_T<SW, true, true, true>(a, rows, st) : launch_csr_T<SW, true, false, true>(a, rows, st);
    const bool vec = ((uintptr_t)a.col % 16 == 0) && (a.w == nullptr || (uintptr_t)a.w % 16 == 0);
    if (a.w != nullptr) return vec ? launch_csr_T<SW, true, true>(a, rows, st) : launch_csr_T<SW, false, true>(a, rows, st);
    return vec ? launch_csr_T<SW, true, false>(a, rows, st) : launch_csr_T<SW, false, false>(a, rows, st);
}

// rows: rows per CTA (1..256); SW: lanes per row.
cudaError_t launch_csr_step(const CsrArgs &a, int SW, int rows, cudaStream_t st) {
    if (rows < 1 || rows > 256) return cudaErrorInvalidValue;
    switch (SW) {
        case 1: return launch_csr_SW<1>(a, rows, st);
        case 2: return launch_csr_SW<2>(a, rows, st);
        case 4: return launch_csr_SW<4>(a, rows, st);
        case 8: return launch_csr_SW<8>(a, rows, st);
        case 16: return launch_csr_SW<16>(a, rows, st);
        case 32: return launch_csr_SW<32>(a, rows, st);
        default: return cudaErrorInvalidValue;
    }
}

// Prefer L1 over shared memory for the V_dend gathers (the kernel uses 1 KB of shared).
template <int SW>
static void carveout_SW() {
    cudaFuncSetAttribute(csr_step_kernel<SW, true, true, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    cudaFuncSetAttribute(csr_step_kernel<SW, false, true, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    cudaFuncSetAttribute(csr_step_kernel<SW, true, false, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    cudaFuncSetAttribute(csr_step_kernel<SW, false, false, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    cudaFuncSetAttribute(csr_step_kernel<SW, true, true, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    cudaFuncSetAttribute(csr_step_kernel<SW, true, false, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    cudaFuncSetAttribute(csr_step_kernel<SW, true, true, true, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    cudaFuncSetAttribute(csr_step_kernel<SW, true, false, true, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
}
cudaError_t prepare_csr_step() {
    carveout_SW<1>();
    carveout_SW<2>();
    carveout_SW<4>();
    carveout_SW<8>();
    carveout_SW<16>();
    carveout_SW<32>();
    return cudaGetLastError();
}

// ---- column-chunked variant: V_dend staged in shared memory -------------------------------
// For large networks the V_dend gathers of a random graph touch a different L1 line per
// lane.  Here the column space is cut into chunks of CSR_CHUNK floats (128 KB); each
// CTA (one per SM, 1024 threads) owns `rows` consecutive rows and, chunk by chunk,
// stages V_dend[chunk] into shared memory with one bulk copy and sums the edges of its
// rows whose columns fall in that chunk (the per-row chunk boundaries are precomputed:
// mid[(c-1) * n + i] is the first edge of row i in chunk c).  The gathers then hit shared
// memory while the indices and weights stream from HBM.
// PAD: the padded layout (a.col16p, a.wp, a.segoff): every (chunk, row) segment is whole
// 16-byte groups of chunk-relative columns, its padding entries index vs[nb + row offset],
// which holds the row's own V_dend (a term with dV = 0, exactly 0); no head or tail edges.
template <int SW, bool VEC, bool HAS_W, bool C16, bool LIN = false, bool PAD = false>
__global__ void __launch_bounds__(1024) csr_chunk_step_kernel(const CsrArgs a, int rows, const int32_t *mid,
                                                              int n_chunks) {
    static_assert(!LIN || C16, "linear junctions run on the 16-bit column layout");
    static_assert(!PAD || C16, "the padded layout has 16-bit columns");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *vs = reinterpret_cast<float *>(smem_raw);
    const int nb = min(CSR_CHUNK, a.c.n_pad);
    float *ic_s = vs + nb + rows;   // vs[nb .. nb + rows): the rows' own V_dend (PAD)
    __shared__ __align__(8) uint64_t bar;
    pdl_enter();
    const StepCommon &c = a.c;
    const int n = c.n;
    const int row0 = blockIdx.x * rows;
    const int64_t t = step_index(c);
    const float *vcur = vd_cur(c);
    float *vnext = vd_next(c);
    const int sub = threadIdx.x / SW, li = threadIdx.x % SW, nsub = blockDim.x / SW;
    const int iters = (rows + nsub - 1) / nsub;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        ic_s[r] = 0.0f;
        if (PAD) vs[nb + r] = row0 + r < n ? vcur[row0 + r] : 0.0f;   // past the chunk: never overwritten
    }
    __syncthreads();
    for (int ch = 0; ch < n_chunks; ++ch) {
        const int c0 = ch * CSR_CHUNK;
        const int len = min(CSR_CHUNK, c.n_pad - c0);
        if (threadIdx.x == 0) {
            mbar_expect_tx(&bar, (uint32_t)len * 4u);
            bulk_g2s(vs, vcur + c0, (uint32_t)len * 4u, &bar);
        }
        const bool landed = mbar_wait_bounded(&bar, (uint32_t)(ch & 1));
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) {
                atomicOr(c.status, (uint32_t)ST_TIMEOUT);
                (void)mbar_wait_bounded(&bar, (uint32_t)(ch & 1));
            }
            return;
        }
        // The bounds of a row's segment in this chunk and its V_dend.  With 16 or more lanes
        // per row (long rows, few rows per group) they are loaded two rows ahead and the
        // next row's index (and weight) stream is requested into L2 one row ahead, so that
        // each row waits on an L2 latency rather than on two HBM latencies.
        auto bounds = [&](int it, int &e0, int &e1, float &vi) {
            const int rr = sub + it * nsub, i = row0 + rr;
            e0 = e1 = 0;
            vi = 0.0f;
            if (it < iters && rr < rows && i < n) {
                if (PAD) {   // chunk-major segments: (ch, i + 1) starts where (ch, i) ends
                    e0 = a.segoff[(int64_t)ch * n + i];
                    e1 = a.segoff[(int64_t)ch * n + i + 1];
                } else {
                    e0 = ch == 0 ? a.row_ptr[i] : mid[(int64_t)(ch - 1) * n + i];
                    e1 = ch == n_chunks - 1 ? a.row_ptr[i + 1] : mid[(int64_t)ch * n + i];
                }
                vi = vcur[i];
            }
        };
        constexpr bool AHEAD = SW >= 16;
        int e0n = 0, e1n = 0, e0m = 0, e1m = 0;
        float vin = 0.0f, vim = 0.0f;
        if (AHEAD) {
            bounds(0, e0n, e1n, vin);
            bounds(1, e0m, e1m, vim);
        }
        for (int it = 0; it < iters; ++it) {
            const int rr = sub + it * nsub;
            int e0, e1;
            float vi;
            if (AHEAD) {
                e0 = e0n;
                e1 = e1n;
                vi = vin;
                e0n = e0m;
                e1n = e1m;
                vin = vim;
                bounds(it + 2, e0m, e1m, vim);
                if (li == 0 && e1n > e0n) {   // the next row's stream, in whole 16-byte groups
                    if (C16) {   // col16 (and col16p) are padded to whole 16-byte groups
                        const int64_t b0 = ((int64_t)e0n * 2) & ~(int64_t)15, b1 = ((int64_t)e1n * 2 + 15) & ~(int64_t)15;
                        bulk_prefetch_l2(reinterpret_cast<const char *>(PAD ? a.col16p : a.col16) + b0,
                                         (uint32_t)(b1 - b0));
                    } else {     // 32-bit columns: the last partial group is left out
                        const int64_t b0 = ((int64_t)e0n * 4) & ~(int64_t)15, b1 = ((int64_t)e1n * 4) & ~(int64_t)15;
                        if (b1 > b0) bulk_prefetch_l2(reinterpret_cast<const char *>(a.col) + b0, (uint32_t)(b1 - b0));
                    }
                    if (HAS_W) {
                        const int64_t b0 = ((int64_t)e0n * 4) & ~(int64_t)15, b1 = ((int64_t)e1n * 4) & ~(int64_t)15;
                        if (b1 > b0)
                            bulk_prefetch_l2(reinterpret_cast<const char *>(PAD ? a.wp : a.w) + b0, (uint32_t)(b1 - b0));
                    }
                }
            } else {
                bounds(it, e0, e1, vi);
            }
            float acc = 0.0f;
            if (e1 > e0) {   // rows past the end (and empty segments) have e0 == e1
                if (PAD)
                    acc = csr_row_sum16<SW, HAS_W, true, LIN, true>(a.col16p, a.wp, e0, e1, vi, li, VjPadded{vs});
                else if (C16)
                    acc = csr_row_sum16<SW, HAS_W, true, LIN>(a.col16, a.w, e0, e1, vi, li, VjChunk{vs});
                else
                    acc = csr_row_sum_smem<SW, VEC, HAS_W>(vs, c0, a.col, a.w, e0, e1, vi, li);
            }
#pragma unroll
            for (int off = SW / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (li == 0 && rr < rows) ic_s[rr] += acc;
        }
        // all reads of this chunk are done before the next bulk copy overwrites it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
    for (int rr = threadIdx.x; rr < rows; rr += blockDim.x) {
        const int i = row0 + rr;
        if (i >= n) break;
        const float ic = (HAS_W ? ic_s[rr] : ic_s[rr] * a.g) * (1.0f / GJ_SCALE);
        const Cell cell = load_cell(c.S, vcur, i);
        float iapp = pulse_current(c.pulses, i, t);
        if (c.iapp != nullptr) iapp += c.iapp[i];
        const CellNext o = cell_step(c.P, cell, ic, iapp);
        finish_cell(c, t, vnext, i, o);
    }
}

// the chunk, the rows' own V_dend (padded layout) and their currents
size_t csr_chunk_smem_bytes(int n_pad, int rows) {
    return (size_t)(n_pad < CSR_CHUNK ? n_pad : CSR_CHUNK) * sizeof(float) + 2 * (size_t)rows * sizeof(float);
}

template <int SW, bool VEC, bool HAS_W, bool C16 = false, bool LIN = false, bool PAD = false>
static cudaError_t chunk_T(const CsrArgs &a, int rows, const int32_t *mid, int n_chunks, bool prepare,
                           cudaStream_t st) {
    const size_t smem = csr_chunk_smem_bytes(a.c.n_pad, rows);
    if (prepare)
        return cudaFuncSetAttribute(csr_chunk_step_kernel<SW, VEC, HAS_W, C16, LIN, PAD>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = (a.c.n + rows - 1) / rows;
    return launch_k(csr_chunk_step_kernel<SW, VEC, HAS_W, C16, LIN, PAD>, dim3(grid), dim3(1024), smem, st,
                    a.c.pdl != 0, a, rows, mid, n_chunks);
}
template <int SW>
static cudaError_t chunk_SW(const CsrArgs &a, int rows, const int32_t *mid, int n_chunks, bool prepare,
                            cudaStream_t st) {
    const bool vec = ((uintptr_t)a.col % 16 == 0) && (a.w == nullptr || (uintptr_t)a.w % 16 == 0);
    if (prepare) {   // set the limit on every instantiation the launch may pick
        cudaError_t e = chunk_T<SW, true, true>(a, rows, mid, n_chunks, true, st);
        if (e == cudaSuccess) e = chunk_T<SW, false, true>(a, rows, mid, n_chunks, true, st);
        if (e == cudaSuccess) e = chunk_T<SW, true, false>(a, rows, mid, n_chunks, true, st);
        if (e == cudaSuccess) e = chunk_T<SW, false, false>(a, rows, mid, n_chunks, true, st);
        if (e == cudaSuccess) e = chunk_T<SW, true, true, true>(a, rows, mid, n_chunks, true, st);
        if (e == cudaSuccess) e = chunk_T<SW, true, false, true>(a, rows, mid, n_chunks, true, st);
        if (e == cudaSuccess) e = chunk_T<SW, true, true, true, true>(a, rows, mid, n_chunks, true, st);
        if (e == cudaSuccess) e = chunk_T<SW, true, false, true, true>(a, rows, mid, n_chunks, true, st);
        if (e == cudaSuccess) e = chunk_T<SW, true, true, true, false, true>(a, rows, mid, n_chunks, true, st);
        if (e == cudaSuccess) e = chunk_T<SW, true, false, true, false, true>(a, rows, mid, n_chunks, true, st);
        if (e == cudaSuccess) e = chunk_T<SW, true, true, true, true, true>(a, rows, mid, n_chunks, true, st);
        if (e == cudaSuccess) e = chunk_T<SW, true, false, true, true, true>(a, rows, mid, n_chunks, true, st);
        return e;
    }
    if (a.col16p != nullptr) {   // the padded layout (weights in a.wp when per edge)
        if (a.lin)
            return a.wp != nullptr ? chunk_T<SW, true, true, true, true, true>(a, rows, mid, n_chunks, false, st)
                                   : chunk_T<SW, true, false, true, true, true>(a, rows, mid, n_chunks, false, st);
        return a.wp != nullptr ? chunk_T<SW, true, true, true, false, true>(a, rows, mid, n_chunks, false, st)
                               : chunk_T<SW, true, false, true, false, true>(a, rows, mid, n_chunks, false, st);
    }
    if (a.lin) {
        if (a.col16 == nullptr) return cudaErrorInvalidValue;
        return a.w != nullptr ? chunk_T<SW, true, true, true, true>(a, rows, mid, n_chunks, false, st)
                              : chunk_T<SW, true, false, true, true>(a, rows, mid, n_chunks, false, st);
    }
    if (a.col16 != nullptr)
        return a.w != nullptr ? chunk_T<SW, true, true, true>(a, rows, mid, n_chunks, false, st)
                              : chunk_T<SW, true, false, true>(a, rows, mid, n_chunks, false, st);
    if (a.w != nullptr)
        return vec ? chunk_T<SW, true, true>(a, rows, mid, n_chunks, false, st)
                   : chunk_T<SW, false, true>(a, rows, mid, n_chunks, false, st);
    return vec ? chunk_T<SW, true, false>(a, rows, mid, n_chunks, false, st)
               : chunk_T<SW, false, false>(a, rows, mid, n_chunks, false, st);
}

// rows: rows per CTA (1..1024); mid: (n_chunks - 1) x n interior chunk boundaries.
cudaError_t launch_csr_chunk_step(const CsrArgs &a, int SW, int rows, const int32_t *mid, int n_chunks, bool prepare,
                                  cudaStream_t st) {
    if (rows < 1 || rows > 1024 || n_chunks < 1) return cudaErrorInvalidValue;
    switch (SW) {
        case 1: return chunk_SW<1>(a, rows, mid, n_chunks, prepare, st);
        case 2: return chunk_SW<2>(a, rows, mid, n_chunks, prepare, st);
        case 4: return chunk_SW<4>(a, rows, mid, n_chunks, prepare, st);
        case 8: return chunk_SW<8>(a, rows, mid, n_chunks, prepare, st);
        case 16: return chunk_SW<16>(a, rows, mid, n_chunks, prepare, st);
        case 32: return chunk_SW<32>(a, rows, mid, n_chunks, prepare, st);
        default: return cudaErrorInvalidValue;
    }
}

// mid[(c - 1) * n + i] = first edge of row i whose column is >= c * CSR_CHUNK (c = 1..C-1)
__global__ void csr_chunk_bounds_kernel(const int32_t *row_ptr, const int32_t *col, int32_t n, int n_chunks,
                                        int32_t *mid) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int ch = 1; ch < n_chunks; ++ch) {
        const int bound = ch * CSR_CHUNK;
        int lo = row_ptr[i], hi = row_ptr[i + 1];   // first e in [lo, hi) with col[e] >= bound
        while (lo < hi) {
            const int m = (lo + hi) >> 1;
            if (col[m] < bound) lo = m + 1;
            else hi = m;
        }
        mid[(int64_t)(ch - 1) * n + i] = lo;
    }
}

// The padded layout from the sorted CSR: one warp per (chunk, row) segment, in chunk-major
// order at off[seg]; columns chunk-relative, then padding entries nb + (i mod rows) (the
// slot of row i's own V_dend in its CTA) up to the next multiple of 8, weight 0.
__global__ void csr_pad_fill_kernel(const int32_t *row_ptr, const int32_t *mid, const int32_t *col, const float *w,
                                    int32_t n, int n_chunks, int rows, int nb, const int32_t *off, uint16_t *col16p,
                                    float *wp) {
    const int64_t seg = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (seg >= (int64_t)n_chunks * n) return;
    const int ch = (int)(seg / n), i = (int)(seg % n);
    const int b = ch == 0 ? row_ptr[i] : mid[(int64_t)(ch - 1) * n + i];
    const int e = ch == n_chunks - 1 ? row_ptr[i + 1] : mid[(int64_t)ch * n + i];
    const int o = off[seg], len = off[seg + 1] - o;
    for (int k = lane; k < len; k += 32) {
        const bool real = k < e - b;
        col16p[o + k] = (uint16_t)(real ? col[b + k] - ch * CSR_CHUNK : nb + i % rows);
        if (wp) wp[o + k] = real ? w[b + k] : 0.0f;
    }
}

cudaError_t launch_csr_pad_fill(const int32_t *row_ptr, const int32_t *mid, const int32_t *col, const float *w,
                                int32_t n, int n_chunks, int rows, int nb, const int32_t *off, uint16_t *col16p,
                                float *wp, cudaStream_t st) {
    const int64_t segs = (int64_t)n_chunks * n;
    csr_pad_fill_kernel<<<(unsigned)((segs + 7) / 8), 256, 0, st>>>(row_ptr, mid, col, w, n, n_chunks, rows, nb, off,
                                                                     col16p, wp);
    return cudaGetLastError();
}

cudaError_t launch_csr_chunk_bounds(const int32_t *row_ptr, const int32_t *col, int32_t n, int n_chunks, int32_t *mid,
                                    cudaStream_t st) {
    if (n_chunks <= 1) return cudaSuccess;
    csr_chunk_bounds_kernel<<<(n + 255) / 256, 256, 0, st>>>(row_ptr, col, n, n_chunks, mid);
    return cudaGetLastError();
}

// ---- simplified gap junctions (SGJ use case, Sec. 2.3.2) ---------------------------------
// Each connection contributes w (V_i - V_j) (the small-dV limit of the RGJ term).
// Dense: Ic_i = g sum_j (V_i - V_j) = g (N (V_i - m) - sum_j (V_j - m)), m = V_dend of cell 0
// (shifted so nearly equal voltages do not cancel).  Larger networks take two launches
// per step: P CTAs write Kahan partial sums of V_j - m over fixed strided ranges, then
// every CTA of the update sums the P partials in index order and updates its cells
// (deterministic).
__global__ void __launch_bounds__(256) sgj_partial_kernel(const StepCommon c, float *part) {
    __shared__ float red[8];
    pdl_enter();
    const int64_t t = step_index(c);
    const float *vcur = vd_cur(c);
    const float m = vcur[0];
    float s = 0.0f, cc = 0.0f;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < c.n; j += (int64_t)gridDim.x * blockDim.x)
        kahan_add(s, cc, vcur[j] - m);
    float v = s - cc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        part[blockIdx.x] = tot;
    }
}
// part == NULL (networks of at most SGJ_ONE_LAUNCH cells): every CTA sums V_j - m over all
// cells itself, in one fixed order (the same in every CTA), so one launch does the step.
__global__ void __launch_bounds__(256) sgj_dense_update_kernel(const StepCommon c, const float *part, int n_part,
                                                               float g) {
    __shared__ float U_sh;
    __shared__ float red[8];
    pdl_enter();
    const int64_t t = step_index(c);
    const float *vcur = vd_cur(c);
    float *vnext = vd_next(c);
    if (part == nullptr) {
        const float m0 = vcur[0];
        float s = 0.0f, cc = 0.0f;
        for (int64_t j = threadIdx.x; j < c.n; j += blockDim.x) kahan_add(s, cc, vcur[j] - m0);
        float v = s - cc;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            float tot = 0.0f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
            U_sh = tot;
        }
    } else if (threadIdx.x == 0) {
        float s = 0.0f, cc = 0.0f;
        for (int q = 0; q < n_part; ++q) kahan_add(s, cc, part[q]);
        U_sh = s - cc;
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n) return;
    const float m = vcur[0];
    const float ic = g * fmaf((float)c.n, vcur[i] - m, -U_sh);
    const Cell cell = load_cell(c.S, vcur, i);
    float iapp = pulse_current(c.pulses, i, t);
    if (c.iapp != nullptr) iapp += c.iapp[i];
    const CellNext o = cell_step(c.P, cell, ic, iapp);
    finish_cell(c, t, vnext, i, o);
}
cudaError_t launch_sgj_dense_step(const StepCommon &c, float g, float *part, cudaStream_t st) {
    if (c.n <= SGJ_ONE_LAUNCH) {
        return launch_k(sgj_dense_update_kernel, dim3((c.n + 255) / 256), dim3(256), 0, st, c.pdl != 0, c,
                        (const float *)nullptr, 0, g);
    }
    const int n_part = sgj_partials(c.n);
    cudaError_t e = launch_k(sgj_partial_kernel, dim3(n_part), dim3(256), 0, st, c.pdl != 0, c, part);
    if (e != cudaSuccess) return e;
    return launch_k(sgj_dense_update_kernel, dim3((c.n + 255) / 256), dim3(256), 0, st, c.pdl != 0, c,
                    (const float *)part, n_part, g);
}
int sgj_partials(int n) { return std::min(256, std::max(1, (n + 4095) / 4096)); }

// CSR: eight lanes per row, 32 rows per CTA, then the cell update of the CTA's rows.
__global__ void __launch_bounds__(256) sgj_csr_step_kernel(const CsrArgs a) {
    __shared__ float ic_s[32];
    pdl_enter();
    const StepCommon &c = a.c;
    const int64_t t = step_index(c);
    const float *vcur = vd_cur(c);
    float *vnext = vd_next(c);
    const int sub = threadIdx.x >> 3, li = threadIdx.x & 7;
    const int i = blockIdx.x * 32 + sub;
    float acc = 0.0f;
    if (i < c.n) {
        const float vi = vcur[i];
        for (int e = a.row_ptr[i] + li; e < a.row_ptr[i + 1]; e += 8) {
            const float dv = vi - __ldg(vcur + __ldg(a.col + e));
            acc = a.w != nullptr ? fmaf(__ldg(a.w + e), dv, acc) : acc + dv;
        }
    }
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (li == 0) ic_s[sub] = a.w != nullptr ? acc : acc * a.g;
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int r = blockIdx.x * 32 + threadIdx.x;
    if (r >= c.n) return;
    const Cell cell = load_cell(c.S, vcur, r);
    float iapp = pulse_current(c.pulses, r, t);
    if (c.iapp != nullptr) iapp += c.iapp[r];
    const CellNext o = cell_step(c.P, cell, ic_s[threadIdx.x], iapp);
    finish_cell(c, t, vnext, r, o);
}
cudaError_t launch_sgj_csr_step(const CsrArgs &a, cudaStream_t st) {
    return launch_k(sgj_csr_step_kernel, dim3((a.c.n + 31) / 32), dim3(256), 0, st, a.c.pdl != 0, a);
}

// ---- half-work CSR (each stored pair evaluated once) ------------------------------------
// The pair term is odd in dV and the weights are symmetric, so the term of the stored edge
// (j, i) is exactly the negated term of (i, j).  Pass 1 walks the upper triangle: for each
// edge e = (i, j), j > i, it adds t_e to row i and writes -t_e into slot[rev[e]], the
// position of the mirrored edge (j, i) in row j (every slot is written by exactly one
// edge: no atomics).  Pass 2 adds to each row the slots of its lower edges, in a fixed
// order, and runs the cell update.  split[i] is the first edge of row i with col > i.
template <int SW, bool HAS_W>
__global__ void __launch_bounds__(256) csr_half_upper_kernel(const CsrArgs a, int rows, const int32_t *split,
                                                             const int32_t *rev, float *slot, float *icu) {
    pdl_enter();
    const StepCommon &c = a.c;
    const float *vcur = vd_cur(c);
    const int sub = threadIdx.x / SW, li = threadIdx.x % SW, nsub = blockDim.x / SW;
    const int row0 = blockIdx.x * rows;
    for (int rr = sub; rr - sub < rows; rr += nsub) {   // the same trip count in every lane
        const int i = row0 + rr;
        float acc = 0.0f;
        if (rr < rows && i < c.n) {
            const float vi = vcur[i];
            for (int e = split[i] + li; e < a.row_ptr[i + 1]; e += SW) {
                const float t = gj_edge(vi, __ldg(vcur + __ldg(a.col + e)), HAS_W ? __ldg(a.w + e) : 1.0f);
                acc += t;
                slot[__ldg(rev + e)] = -t;
            }
        }
#pragma unroll
        for (int off = SW / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (li == 0 && rr < rows && i < c.n) icu[i] = acc;
    }
}

template <int SW, bool HAS_W>
__global__ void __launch_bounds__(256) csr_half_lower_kernel(const CsrArgs a, int rows, const int32_t *split,
                                                             const float *slot, const float *icu) {
    __shared__ float ic_s[256];
    pdl_enter();
    const StepCommon &c = a.c;
    const int64_t t = step_index(c);
    const float *vcur = vd_cur(c);
    float *vnext = vd_next(c);
    const int sub = threadIdx.x / SW, li = threadIdx.x % SW, nsub = blockDim.x / SW;
    const int row0 = blockIdx.x * rows;
    for (int rr = sub; rr - sub < rows; rr += nsub) {
        const int i = row0 + rr;
        float acc = 0.0f;
        if (rr < rows && i < c.n)
            for (int e = a.row_ptr[i] + li; e < split[i]; e += SW) acc += slot[e];
#pragma unroll
        for (int off = SW / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (li == 0 && rr < rows && i < c.n) {
            const float tot = icu[i] + acc;
            ic_s[rr] = (HAS_W ? tot : tot * a.g) * (1.0f / GJ_SCALE);
        }
    }
    __syncthreads();
    if ((int)threadIdx.x >= rows) return;
    const int i = row0 + threadIdx.x;
    if (i >= c.n) return;
    const Cell cell = load_cell(c.S, vcur, i);
    float iapp = pulse_current(c.pulses, i, t);
    if (c.iapp != nullptr) iapp += c.iapp[i];
    const CellNext o = cell_step(c.P, cell, ic_s[threadIdx.x], iapp);
    finish_cell(c, t, vnext, i, o);
}

template <int SW>
static cudaError_t half_SW(const CsrArgs &a, int rows, const int32_t *split, const int32_t *rev, float *slot,
                           float *icu, cudaStream_t st) {
    const int grid = (a.c.n + rows - 1) / rows;
    const bool pdl = a.c.pdl != 0;
    cudaError_t e = a.w != nullptr
                        ? launch_k(csr_half_upper_kernel<SW, true>, dim3(grid), dim3(256), 0, st, pdl, a, rows, split, rev, slot, icu)
                        : launch_k(csr_half_upper_kernel<SW, false>, dim3(grid), dim3(256), 0, st, pdl, a, rows, split, rev, slot, icu);
    if (e != cudaSuccess) return e;
    const float *cslot = slot, *cicu = icu;
    return a.w != nullptr
               ? launch_k(csr_half_lower_kernel<SW, true>, dim3(grid), dim3(256), 0, st, pdl, a, rows, split, cslot, cicu)
               : launch_k(csr_half_lower_kernel<SW, false>, dim3(grid), dim3(256), 0, st, pdl, a, rows, split, cslot, cicu);
}

// Both passes of a half-work CSR step (rows per CTA <= 256; SW lanes per row).
cudaError_t launch_csr_half_step(const CsrArgs &a, int SW, int rows, const int32_t *split, const int32_t *rev,
                                 float *slot, float *icu, cudaStream_t st) {
    if (rows < 1 || rows > 256) return cudaErrorInvalidValue;
    switch (SW) {
        case 1: return half_SW<1>(a, rows, split, rev, slot, icu, st);
        case 2: return half_SW<2>(a, rows, split, rev, slot, icu, st);
        case 4: return half_SW<4>(a, rows, split, rev, slot, icu, st);
        case 8: return half_SW<8>(a, rows, split, rev, slot, icu, st);
        case 16: return half_SW<16>(a, rows, split, rev, slot, icu, st);
        case 32: return half_SW<32>(a, rows, split, rev, slot, icu, st);
        default: return cudaErrorInvalidValue;
    }
}

// ---- compact column layout: the low 16 bits of every column (zero padding to 8 entries)
__global__ void csr_col16_kernel(const int32_t *col, int64_t nnz, int64_t n_alloc, uint16_t *col16) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_alloc) col16[e] = e < nnz ? (uint16_t)((uint32_t)col[e] & 0xFFFFu) : (uint16_t)0;
}
cudaError_t launch_csr_col16(const int32_t *col, int64_t nnz, int64_t n_alloc, uint16_t *col16, cudaStream_t st) {
    if (n_alloc <= 0) return cudaSuccess;
    csr_col16_kernel<<<(unsigned)((n_alloc + 255) / 256), 256, 0, st>>>(col, nnz, n_alloc, col16);
    return cudaGetLastError();
}

// ---- stand-alone cell update (no gap junctions, or Ic computed by another launch) ----
__global__ void __launch_bounds__(256) cell_step_kernel(const CellArgs a) {
    pdl_enter();
    const StepCommon &c = a.c;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n) return;
    const int64_t t = step_index(c);
    const float *vcur = vd_cur(c);
    float *vnext = vd_next(c);
    const Cell cell = load_cell(c.S, vcur, i);
    const float ic = a.ic != nullptr ? a.ic[i] : 0.0f;
    float iapp = pulse_current(c.pulses, i, t);
    if (c.iapp != nullptr) iapp += c.iapp[i];
    const CellNext o = a.cellp != nullptr ? cell_step(cell_model(c.P, a.cellp, c.S.stride, i), cell, ic, iapp)
                                          : cell_step(c.P, cell, ic, iapp);
    finish_cell(c, t, vnext, i, o);
}

cudaError_t launch_cell_step(const CellArgs &a, cudaStream_t st) {
    const int64_t grid = ((int64_t)a.c.n + 255) / 256;
    return launch_k(cell_step_kernel, dim3((unsigned)grid), dim3(256), 0, st, a.c.pdl != 0, a);
}

// ---- rate functions and default state (host-visible copies of the device model) ----
__global__ void rates_kernel(float V, float ca, float *out) {
    if (threadIdx.x != 0) return;
    const Rate g[NG] = {rate_r(V), rate_s(ca), rate_q(V), rate_k(V), rate_l(V), {minf_na(V), 0.0f},
                        rate_hs(V), rate_ns(V), rate_x(V), {minf_na(V), 0.0f}, rate_ha(V), rate_x(V)};
    for (int k = 0; k < NG; ++k) {
        out[k] = g[k].xinf;
        out[NG + k] = g[k].inv_tau > 0.0f ? 1.0f / g[k].inv_tau : 0.0f;
    }
}

cudaError_t launch_rates(float V, float ca, float *out, cudaStream_t st) {
    rates_kernel<<<1, 32, 0, st>>>(V, ca, out);
    return cudaGetLastError();
}

__global__ void default_state_kernel(ModelF P, float V0, float ca0, float gcal, int32_t n, int64_t stride, float *S) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float r = rate_r(V0).xinf;
    const float v[NF] = {V0, V0, V0, ca0, r, rate_s(ca0).xinf, rate_q(V0).xinf, rate_k(V0).xinf,
                         rate_l(V0).xinf, minf_na(V0), rate_hs(V0).xinf, rate_ns(V0).xinf, rate_x(V0).xinf,
                         minf_na(V0), rate_ha(V0).xinf, rate_x(V0).xinf, gcal, P.gCaH * r * r * (V0 - P.VCa), 0.0f};
    for (int f = 0; f < NF; ++f) S[f * stride + i] = v[f];
}

cudaError_t launch_default_state(const ModelF &P, float V0, float ca0, float gcal, int32_t n, int64_t stride,
                                 float *state, cudaStream_t st) {
    default_state_kernel<<<(n + 255) / 256, 256, 0, st>>>(P, V0, ca0, gcal, n, stride, state);
    return cudaGetLastError();
}

// ---- small helpers ------------------------------------------------------------------
__global__ void advance_kernel(int64_t *t_dev, int64_t k) { *t_dev += k; }

cudaError_t launch_advance(int64_t *t_dev, int64_t k, cudaStream_t st) {
    advance_kernel<<<1, 1, 0, st>>>(t_dev, k);
    return cudaGetLastError();
}

__global__ void fill_kernel(float *p, float v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

cudaError_t launch_fill(float *p, float v, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(p, v, n);
    return cudaGetLastError();
}

}  // namespace ion
