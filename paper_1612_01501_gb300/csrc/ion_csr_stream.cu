// ion_csr_stream.cu -- CSR step for networks whose connectivity streams from HBM, with the
// index stream moved by bulk asynchronous copies.
//
// Algorithm 1 over a programmed weight matrix (Sec. 2.3), as in ion_csr.cu.  When the
// CSR does not fit in L2 every step reads it from HBM once, and the kernel must keep
// enough bytes in flight to cover HBM latency.  Here the connectivity is re-laid out once,
// chunk-major: the columns are cut into chunks of CSR_SCHUNK cells and, for each chunk,
// the edges of row 0, row 1, ... whose columns fall in it are stored contiguously as
// 16-bit chunk-relative columns (crp[c][i] = first edge of row i in chunk c).  A CTA owns
// `rows` consecutive rows and walks (chunk, batch of 32 rows) items in order:
//   - V_dend of the chunk is bulk-copied into one of two shared-memory buffers (the next
//     chunk lands while the current one is in use);
//   - the edges of a batch (one contiguous range of the chunk-major arrays) are
//     bulk-copied into one of NS ring slots, NS items ahead of their use, so a few tens
//     of KB per SM are in flight while the warps compute;
//   - warp w sums the edges of row 32k + w: column from the slot, V_dend from the chunk
//     buffer (both in shared memory), and adds the sum to the row's current in chunk
//     order (deterministic).
// Thread 0 issues every copy; completion is counted in bytes on one mbarrier per buffer,
// every wait is bounded.  After the last item each thread runs the explicit-Euler update
// of its row (the row's state was loaded at kernel start).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ion.h"
#include "ion_async.cuh"
#include "ion_csr_core.cuh"
#include "ion_kernels.cuh"
#include "ion_sim.h"

namespace ion {

constexpr int STREAM_BATCH = 32;          // rows per item (one warp per row)
constexpr int STREAM_MAX_SLOTS = 4;
constexpr int STREAM_SMEM = 220 * 1024;   // dynamic shared memory budget per CTA

struct CsrStreamArgs {
    StepCommon c;
    const int32_t *crp;     // [nc][n + 1] first edge of each row in each chunk (chunk-major positions)
    const uint16_t *ccol;   // chunk-relative columns, chunk-major, padded by 8 entries
    const float *cw;        // weights in the same order (padded), or NULL: every weight is g
    float g;
    int32_t nc;             // chunks
    int32_t rows;           // rows per CTA (a multiple of STREAM_BATCH, <= 1024)
    int32_t slot_edges;     // capacity of one ring slot (a multiple of 8)
    int32_t n_slots;        // ring slots (2..STREAM_MAX_SLOTS)
};

struct StreamSmem {
    float *vbuf[2];
    uint16_t *es;    // [n_slots][slot_edges]
    float *ws;       // [n_slots][slot_edges] or NULL
    int32_t *rp;     // [nc][rows + 1] row bounds of this CTA's rows
    float *vi;       // [rows] V_dend of this CTA's rows
    float *ic;       // [rows] accumulated gap current (scaled)
};

__host__ __device__ inline size_t stream_smem_bytes(int nc, int rows, int se, int ns, bool has_w) {
    return (size_t)2 * CSR_SCHUNK * sizeof(float) + (size_t)ns * se * (sizeof(uint16_t) + (has_w ? sizeof(float) : 0)) +
           (size_t)nc * (rows + 1) * sizeof(int32_t) + (size_t)2 * rows * sizeof(float) + 64;
}

__device__ inline StreamSmem stream_smem(unsigned char *raw, int nc, int rows, int se, int ns, bool has_w) {
    StreamSmem m;
    float *f = reinterpret_cast<float *>(raw);
    m.vbuf[0] = f;
    m.vbuf[1] = f + CSR_SCHUNK;
    unsigned char *p = raw + (size_t)2 * CSR_SCHUNK * sizeof(float);
    m.ws = nullptr;
    if (has_w) {
        m.ws = reinterpret_cast<float *>(p);
        p += (size_t)ns * se * sizeof(float);
    }
    m.es = reinterpret_cast<uint16_t *>(p);
    p += (size_t)ns * se * sizeof(uint16_t);
    p = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
    m.rp = reinterpret_cast<int32_t *>(p);
    p += (size_t)nc * (rows + 1) * sizeof(int32_t);
    m.vi = reinterpret_cast<float *>(p);
    m.ic = m.vi + rows;
    return m;
}

template <bool HAS_W>
__global__ void __launch_bounds__(1024) csr_stream_kernel(const CsrStreamArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t vbar[2], ebar[STREAM_MAX_SLOTS];
    const StepCommon &c = a.c;
    const int n = c.n, rows = a.rows, nc = a.nc, SE = a.slot_edges, NS = a.n_slots;
    const int row0 = blockIdx.x * rows;
    const int nrow = min(rows, n - row0);                 // rows of this CTA that exist
    const int nb = (nrow + STREAM_BATCH - 1) / STREAM_BATCH;
    const int items = nc * nb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = step_index(c);
    const float *vcur = vd_cur(c, t);
    float *vnext = vd_next(c, t);
    const StreamSmem sm = stream_smem(smem_raw, nc, rows, SE, NS, HAS_W);

    // this thread's row for the cell update: its state loads overlap the whole gap sum
    const bool upd = (int)threadIdx.x < nrow;
    Cell cell{};
    if (upd) cell = load_cell(c.S, vcur, row0 + threadIdx.x);

    if (threadIdx.x == 0) {
        mbar_init(&vbar[0], 1);
        mbar_init(&vbar[1], 1);
        for (int q = 0; q < NS; ++q) mbar_init(&ebar[q], 1);
        fence_mbar_init();
    }
    for (int q = threadIdx.x; q < nc * (nrow + 1); q += blockDim.x) {
        const int ch = q / (nrow + 1), r = q % (nrow + 1);
        sm.rp[ch * (rows + 1) + r] = __ldg(a.crp + (int64_t)ch * (n + 1) + row0 + r);
    }
    for (int r = threadIdx.x; r < nrow; r += blockDim.x) {
        sm.vi[r] = vcur[row0 + r];
        sm.ic[r] = 0.0f;
    }
    __syncthreads();

    // producer (thread 0): the copies of V_dend chunk ch and of item m
    auto issue_v = [&](int ch) {
        const int c0 = ch * CSR_SCHUNK;
        const int len = min(CSR_SCHUNK, c.n_pad - c0);
        mbar_expect_tx(&vbar[ch & 1], (uint32_t)len * 4u);
        bulk_g2s(sm.vbuf[ch & 1], vcur + c0, (uint32_t)len * 4u, &vbar[ch & 1]);
    };
    auto item_range = [&](int m, int &e0a, int &e1a) {
        const int ch = m / nb, k = m % nb;
        const int32_t *rp = sm.rp + ch * (rows + 1);
        e0a = rp[k * STREAM_BATCH] & ~7;
        e1a = (rp[min((k + 1) * STREAM_BATCH, nrow)] + 7) & ~7;
    };
    auto issue_e = [&](int m) {
        int e0a, e1a;
        item_range(m, e0a, e1a);
        const int slot = m % NS;
        const uint32_t ne = (uint32_t)(e1a - e0a);
        mbar_expect_tx(&ebar[slot], ne * (uint32_t)(sizeof(uint16_t) + (HAS_W ? sizeof(float) : 0)));
        if (ne > 0) {
            bulk_g2s(sm.es + (size_t)slot * SE, a.ccol + e0a, ne * (uint32_t)sizeof(uint16_t), &ebar[slot]);
            if (HAS_W) bulk_g2s(sm.ws + (size_t)slot * SE, a.cw + e0a, ne * (uint32_t)sizeof(float), &ebar[slot]);
        }
    };
    int v_issued = 0, e_issued = 0;   // thread 0's counts of copies issued
    if (threadIdx.x == 0) {
        for (; v_issued < min(2, nc); ++v_issued) issue_v(v_issued);
        for (; e_issued < min(NS, items); ++e_issued) issue_e(e_issued);
    }

    bool ok = true;
    int m = 0;
    for (; m < items; ++m) {
        const int ch = m / nb, k = m % nb, slot = m % NS;
        bool landed = true;
        if (k == 0) landed = mbar_wait_bounded(&vbar[ch & 1], (uint32_t)((ch >> 1) & 1));
        landed = landed && mbar_wait_bounded(&ebar[slot], (uint32_t)((m / NS) & 1));
        if (__syncthreads_or(!landed)) {
            ok = false;
            break;
        }
        const int r = k * STREAM_BATCH + warp;
        if (warp < STREAM_BATCH && r < nrow) {
            const int32_t *rp = sm.rp + ch * (rows + 1);
            const int e0a = rp[k * STREAM_BATCH] & ~7;
            const int s0 = rp[r] - e0a, s1 = rp[r + 1] - e0a;
            const uint16_t *es = sm.es + (size_t)slot * SE;
            const float *ws = HAS_W ? sm.ws + (size_t)slot * SE : nullptr;
            const float *vs = sm.vbuf[ch & 1];
            const float vi = sm.vi[r];
            float acc = 0.0f;
            int e = s0 + lane;
            for (; e + 96 < s1; e += 128) {   // four gathers in flight per lane
                const float v0 = vs[es[e]], v1 = vs[es[e + 32]], v2 = vs[es[e + 64]], v3 = vs[es[e + 96]];
                const float w0 = HAS_W ? ws[e] : 1.0f, w1 = HAS_W ? ws[e + 32] : 1.0f;
                const float w2 = HAS_W ? ws[e + 64] : 1.0f, w3 = HAS_W ? ws[e + 96] : 1.0f;
                acc += (gj_edge(vi, v0, w0) + gj_edge(vi, v1, w1)) + (gj_edge(vi, v2, w2) + gj_edge(vi, v3, w3));
            }
            for (; e < s1; e += 32) acc += gj_edge(vi, vs[es[e]], HAS_W ? ws[e] : 1.0f);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) sm.ic[r] += acc;
        }
        // every read of this slot (and, after a chunk's last batch, of its V_dend buffer) is
        // done (barrier) before the issuing thread hands the buffer to the async proxy
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if (e_issued < items) issue_e(e_issued++);
            if (k == nb - 1 && v_issued < nc) issue_v(v_issued++);
        }
    }
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicOr(c.status, (uint32_t)ST_TIMEOUT);
            // wait (bounded) for every copy still in flight before the CTA exits
            const int ch = m / nb;
            for (int q = ch; q < v_issued; ++q) (void)mbar_wait_bounded(&vbar[q & 1], (uint32_t)((q >> 1) & 1));
            for (int q = m; q < e_issued; ++q) (void)mbar_wait_bounded(&ebar[q % NS], (uint32_t)((q / NS) & 1));
        }
        return;
    }
    if (!upd) return;
    const int i = row0 + threadIdx.x;
    const float ic = (HAS_W ? sm.ic[threadIdx.x] : sm.ic[threadIdx.x] * a.g) * (1.0f / GJ_SCALE);
    float iapp = pulse_current(c.pulses, i, t);
    if (c.iapp != nullptr) iapp += c.iapp[i];
    const CellNext o = cell_step(c.P, cell, ic, iapp);
    finish_cell(c, t, vnext, i, o);
}

// ---- building the chunk-major layout (device) ---------------------------------------
// cnt[ch * n + i] = edges of row i with column in chunk ch
__global__ void stream_count_kernel(const int32_t *row_ptr, const int32_t *col, int32_t n, int nc, int32_t *cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = row_ptr[i];
    const int end = row_ptr[i + 1];
    for (int ch = 0; ch < nc; ++ch) {
        const int bound = (ch + 1) * CSR_SCHUNK;   // first e in [lo, end) with col[e] >= bound
        int a = lo, b = end;
        while (a < b) {
            const int mid = (a + b) >> 1;
            if (col[mid] < bound) a = mid + 1;
            else b = mid;
        }
        cnt[(int64_t)ch * n + i] = a - lo;
        lo = a;
    }
}
// one warp per row: copy the row's run of each chunk to its chunk-major place
__global__ void stream_scatter_kernel(const int32_t *row_ptr, const int32_t *col, const float *w, int32_t n, int nc,
                                      const int32_t *crp, uint16_t *ccol, float *cw) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= n) return;
    const int i = (int)gw;
    int src = row_ptr[i];
    for (int ch = 0; ch < nc; ++ch) {
        const int dst = crp[(int64_t)ch * (n + 1) + i];
        const int len = crp[(int64_t)ch * (n + 1) + i + 1] - dst;
        for (int q = lane; q < len; q += 32) {
            ccol[dst + q] = (uint16_t)(col[src + q] - ch * CSR_SCHUNK);
            if (cw) cw[dst + q] = w[src + q];
        }
        src += len;
    }
}

}  // namespace ion

using namespace ion;

// Build the chunk-major layout and choose the ring (host-copied, validated CSR only).
// Returns ION_OK with s->stream_ns = 0 when the layout does not apply (the caller then
// uses the row-major staged kernel).
ion_status ion_setup_csr_stream(ion_sim *s) {
    s->stream_ns = 0;
    if (!s->own_csr || s->d_col16 == nullptr || s->nnz <= 0) return ION_OK;
    const int n = s->n;
    const int nc = (s->n_pad + CSR_SCHUNK - 1) / CSR_SCHUNK;
    int rows = (n + s->sms - 1) / s->sms;
    rows = (rows + STREAM_BATCH - 1) / STREAM_BATCH * STREAM_BATCH;
    if (rows > 1024 || (int64_t)nc * (rows + 1) > 4096) return ION_OK;   // per-CTA row bounds must fit
    const bool has_w = s->d_w != nullptr;
    std::vector<int32_t> crp((size_t)nc * (n + 1));
    int32_t *d_cnt = nullptr;
    cudaError_t e = cudaMalloc(&d_cnt, (size_t)nc * n * sizeof(int32_t));
    if (e == cudaSuccess) {
        stream_count_kernel<<<(n + 255) / 256, 256, 0, s->st>>>(s->d_rowptr, s->d_col, n, nc, d_cnt);
        e = cudaGetLastError();
    }
    std::vector<int32_t> cnt((size_t)nc * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_cnt, cnt.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    cudaFree(d_cnt);
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "CSR stream layout: %s", cudaGetErrorString(e));
    int64_t pos = 0;
    for (int ch = 0; ch < nc; ++ch) {
        for (int i = 0; i < n; ++i) {
            crp[(size_t)ch * (n + 1) + i] = (int32_t)pos;
            pos += cnt[(size_t)ch * n + i];
        }
        crp[(size_t)ch * (n + 1) + n] = (int32_t)pos;
    }
    if (pos != s->nnz) return ion_fail(nullptr, ION_ERR_BAD_CSR, "CSR stream layout: edge count mismatch");
    // widest batch (aligned to 8 edges at both ends) over every CTA, chunk and batch
    int64_t span = 8;
    for (int row0 = 0; row0 < n; row0 += rows) {
        const int nrow = std::min(rows, n - row0);
        for (int ch = 0; ch < nc; ++ch)
            for (int k = 0; k * STREAM_BATCH < nrow; ++k) {
                const int32_t *rp = crp.data() + (size_t)ch * (n + 1) + row0;
                const int64_t a0 = rp[k * STREAM_BATCH] & ~7;
                const int64_t a1 = (rp[std::min((k + 1) * STREAM_BATCH, nrow)] + 7) & ~7;
                span = std::max(span, a1 - a0);
            }
    }
    const int se = (int)((span + 7) / 8 * 8);
    int ns = STREAM_MAX_SLOTS;
    while (ns >= 2 && stream_smem_bytes(nc, rows, se, ns, has_w) > (size_t)STREAM_SMEM) --ns;
    if (ns < 2) return ION_OK;
    const size_t smem = stream_smem_bytes(nc, rows, se, ns, has_w);
    e = cudaFuncSetAttribute(has_w ? csr_stream_kernel<true> : csr_stream_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t alloc = s->nnz + 8;
    if (e == cudaSuccess && !s->d_crp) e = cudaMalloc(&s->d_crp, crp.size() * sizeof(int32_t));
    if (e == cudaSuccess && !s->d_ccol) e = cudaMalloc(&s->d_ccol, (size_t)alloc * sizeof(uint16_t));
    if (e == cudaSuccess && has_w && !s->d_cw) e = cudaMalloc(&s->d_cw, (size_t)alloc * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_crp, crp.data(), crp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_ccol, 0, (size_t)alloc * sizeof(uint16_t), s->st);
    if (e == cudaSuccess && has_w) e = cudaMemsetAsync(s->d_cw, 0, (size_t)alloc * sizeof(float), s->st);
    if (e == cudaSuccess) {
        const int64_t threads = (int64_t)n * 32;
        stream_scatter_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s->st>>>(
            s->d_rowptr, s->d_col, s->d_w, n, nc, s->d_crp, s->d_ccol, has_w ? s->d_cw : nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "CSR stream layout: %s", cudaGetErrorString(e));
    s->stream_nc = nc;
    s->stream_rows = rows;
    s->stream_se = se;
    s->stream_ns = ns;
    s->stream_smem = smem;
    return ION_OK;
}

cudaError_t launch_csr_stream(const ion_sim *s, const StepCommon &c, cudaStream_t st) {
    CsrStreamArgs a{};
    a.c = c;
    a.crp = s->d_crp;
    a.ccol = s->d_ccol;
    a.cw = s->d_w ? s->d_cw : nullptr;
    a.g = s->g;
    a.nc = s->stream_nc;
    a.rows = s->stream_rows;
    a.slot_edges = s->stream_se;
    a.n_slots = s->stream_ns;
    const int grid = (s->n + a.rows - 1) / a.rows;
    if (a.cw) csr_stream_kernel<true><<<grid, 1024, s->stream_smem, st>>>(a);
    else csr_stream_kernel<false><<<grid, 1024, s->stream_smem, st>>>(a);
    return cudaGetLastError();
}
