// ion_batch.cu -- many independent networks advanced by one launch per time step.
//
// Parameter sweeps run many small networks of uneven sizes and densities.  Each network
// b gets a segment of the state arrays starting at seg_b (a multiple of 256 cells, the
// tail padded like a single network's V_dend), so dense networks can stage their V_dend
// with one 16-byte aligned bulk copy and CSR networks use global column indices into the
// same arrays.  The work of a step is a list of tiles (network, first row, rows): a
// dense tile is 8 warps x R rows of one network against all of that network's columns
// (the single-network pair loop, ion_dense_core.cuh), a CSR tile is up to 256 rows with
// SW lanes per row (ion_csr_core.cuh); every tile then runs the explicit-Euler update
// of its rows.  Tiles are ordered by decreasing cost so the hardware scheduler packs the
// long ones first; the launches of K steps are captured into one CUDA graph and
// replayed.  ion_autotune times the tile shapes and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "ion.h"
#include "ion_csr_core.cuh"
#include "ion_dense_core.cuh"
#include "ion_kernels.cuh"
#include "ion_sim.h"

namespace ion {

enum TileKind : int32_t { TILE_DENSE = 0, TILE_CSR = 1 };
// CSR tile modes: every weight of the network equals T.g; 16-bit network-local columns
// (col16); the network's V_dend staged in shared memory (with TILE_C16)
enum TileMode : int32_t { TILE_UNIFORM_W = 1, TILE_C16 = 2, TILE_STAGE_V = 4 };

struct BatchTile {
    int32_t kind;
    int32_t seg;     // first cell of the network's segment
    int32_t n;       // cells of the network
    int32_t n_pad;   // padded length of the segment (multiple of 256)
    int32_t row0;    // first row (global cell index) of the tile
    int32_t rows;    // rows of the tile
    int32_t sw;      // CSR: lanes per row
    float g;         // dense: pair weight; CSR with TILE_UNIFORM_W: every edge weight
    int32_t mode;    // CSR: TileMode bits
};

struct BatchArgs {
    StepCommon c;    // c.n = padded total, c.S = state over the padded index space
    const BatchTile *tiles;
    const int32_t *row_ptr;   // padded-index CSR of every CSR network (other rows empty)
    const int32_t *col;
    const uint16_t *col16;    // network-local columns (TILE_C16 networks)
    const float *w;
    int32_t kahan;
};

// V_dend of a network-local column from shared memory (the network's staged copy)
struct VjShared {
    const float *vs;
    __device__ __forceinline__ float operator()(uint32_t j) const { return vs[j]; }
};

// CSR rows of a TILE_C16 tile: 16-bit local columns, V_dend from `vj` (staged or global)
template <int SW, bool HAS_W, class VJ>
__device__ __forceinline__ void batch_csr_rows16(const BatchArgs &a, const BatchTile &T, const float *vcur, VJ vj,
                                                 float *ic_s) {
    const int sub = threadIdx.x / SW, li = threadIdx.x % SW, nsub = blockDim.x / SW;
    const int iters = (T.rows + nsub - 1) / nsub;
    int e0n = 0, e1n = 0;   // the next row's bounds and V_dend, loaded one row ahead
    float vin = 0.0f;
    if (sub < T.rows) {
        e0n = a.row_ptr[T.row0 + sub];
        e1n = a.row_ptr[T.row0 + sub + 1];
        vin = vcur[T.row0 + sub];
    }
    for (int it = 0; it < iters; ++it) {
        const int rr = sub + it * nsub;
        const int e0 = e0n, e1 = e1n;
        const float vi = vin;
        if (rr + nsub < T.rows) {
            e0n = a.row_ptr[T.row0 + rr + nsub];
            e1n = a.row_ptr[T.row0 + rr + nsub + 1];
            vin = vcur[T.row0 + rr + nsub];
        }
        float acc = 0.0f;
        if (rr < T.rows) acc = csr_row_sum16<SW, HAS_W, false>(a.col16, a.w, e0, e1, vi, li, vj);
#pragma unroll
        for (int off = SW / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (li == 0 && rr < T.rows) ic_s[rr] = (HAS_W ? acc : acc * T.g) * (1.0f / GJ_SCALE);
    }
}
template <int SW, class VJ>
__device__ __forceinline__ void batch_csr_rows16_w(const BatchArgs &a, const BatchTile &T, const float *vcur, VJ vj,
                                                   float *ic_s) {
    if (T.mode & TILE_UNIFORM_W) batch_csr_rows16<SW, false>(a, T, vcur, vj, ic_s);
    else batch_csr_rows16<SW, true>(a, T, vcur, vj, ic_s);
}
template <class VJ>
__device__ __forceinline__ void batch_csr_tile16(const BatchArgs &a, const BatchTile &T, const float *vcur, VJ vj,
                                                 float *ic_s) {
    switch (T.sw) {
        case 1: batch_csr_rows16_w<1>(a, T, vcur, vj, ic_s); break;
        case 2: batch_csr_rows16_w<2>(a, T, vcur, vj, ic_s); break;
        case 4: batch_csr_rows16_w<4>(a, T, vcur, vj, ic_s); break;
        case 8: batch_csr_rows16_w<8>(a, T, vcur, vj, ic_s); break;
        case 16: batch_csr_rows16_w<16>(a, T, vcur, vj, ic_s); break;
        default: batch_csr_rows16_w<32>(a, T, vcur, vj, ic_s); break;
    }
}

template <int SW>
__device__ __forceinline__ void batch_csr_rows(const BatchArgs &a, const BatchTile &T, const float *vcur, float *ic_s) {
    const int sub = threadIdx.x / SW, li = threadIdx.x % SW, nsub = blockDim.x / SW;
    const int iters = (T.rows + nsub - 1) / nsub;
    const bool vec = ((uintptr_t)a.col % 16 == 0) && ((uintptr_t)a.w % 16 == 0);
    int e0n = 0, e1n = 0;   // the next row's bounds and V_dend, loaded one row ahead
    float vin = 0.0f;
    if (sub < T.rows) {
        e0n = a.row_ptr[T.row0 + sub];
        e1n = a.row_ptr[T.row0 + sub + 1];
        vin = vcur[T.row0 + sub];
    }
    for (int it = 0; it < iters; ++it) {
        const int rr = sub + it * nsub;
        const int e0 = e0n, e1 = e1n;
        const float vi = vin;
        if (rr + nsub < T.rows) {
            e0n = a.row_ptr[T.row0 + rr + nsub];
            e1n = a.row_ptr[T.row0 + rr + nsub + 1];
            vin = vcur[T.row0 + rr + nsub];
        }
        float acc = 0.0f;
        if (rr < T.rows)
            acc = vec ? csr_row_sum<SW, true, true>(vcur, a.col, a.w, e0, e1, vi, li)
                      : csr_row_sum<SW, false, true>(vcur, a.col, a.w, e0, e1, vi, li);
#pragma unroll
        for (int off = SW / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (li == 0 && rr < T.rows) ic_s[rr] = acc * (1.0f / GJ_SCALE);
    }
}

// 256 threads: 8 warps.  Dense tiles: 8 row groups of R rows, one column split.
template <int R>
__global__ void __launch_bounds__(256) batch_step_kernel(const BatchArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float red_s[32], red_c[32];
    __shared__ float U_sh;
    __shared__ float ic_s[256];
    pdl_enter();

    const BatchTile T = a.tiles[blockIdx.x];
    const StepCommon &c = a.c;
    const int64_t t = step_index(c);
    const float *vcur = vd_cur(c);
    float *vnext = vd_next(c);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (T.kind == TILE_DENSE) {
        const DenseSmem sm = dense_smem(smem_raw, T.n_pad);   // one tile: n_pad <= 8192
        const float *net_v = vcur + T.seg;
        if (threadIdx.x == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) issue_tile(sm, net_v, T.n_pad, 0, bar);
        const float m_shift = net_v[0];
        float ui[R];
        const int local0 = T.row0 - T.seg;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int li = local0 + warp * R + r;
            ui[r] = (warp * R + r < T.rows) ? (net_v[li] - m_shift) * GJ_SCALE : 0.0f;
        }
        uint32_t uses[2] = {0u, 0u};
        float tot[R], Us, Uc;
        if (!gj_pass<R, 1>(sm, net_v, T.n, T.n_pad, bar, uses, m_shift, ui, 0, lane, a.kahan, tot, Us, Uc)) {
            if (threadIdx.x == 0) {
                atomicOr(c.status, (uint32_t)ST_TIMEOUT);
                (void)mbar_wait_bounded(&bar[0], uses[0] & 1u);
            }
            return;
        }
        const float U = gj_reduce<R, 1>(sm, tot, Us, Uc, warp, 0, lane, red_s, red_c, &U_sh);
        if ((int)threadIdx.x < T.rows) {
            const int rr = threadIdx.x;
            ic_s[rr] = row_current<1>(sm, rr, (net_v[local0 + rr] - m_shift) * GJ_SCALE, T.n, U, T.g);
        }
    } else if (T.mode & TILE_STAGE_V) {
        // the network's V_dend (n_pad <= TJ floats) in shared memory, 16-bit local columns
        float *vs = reinterpret_cast<float *>(smem_raw);
        if (threadIdx.x == 0) {
            mbar_init(&bar[0], 1);
            fence_mbar_init();
            mbar_expect_tx(&bar[0], (uint32_t)T.n_pad * 4u);
            bulk_g2s(vs, vcur + T.seg, (uint32_t)T.n_pad * 4u, &bar[0]);
        }
        __syncthreads();
        const bool landed = mbar_wait_bounded(&bar[0], 0u);
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) {
                atomicOr(c.status, (uint32_t)ST_TIMEOUT);
                (void)mbar_wait_bounded(&bar[0], 0u);
            }
            return;
        }
        batch_csr_tile16(a, T, vcur, VjShared{vs}, ic_s);
    } else if (T.mode & TILE_C16) {
        batch_csr_tile16(a, T, vcur, VjGlobal{vcur + T.seg}, ic_s);
    } else {
        switch (T.sw) {
            case 1: batch_csr_rows<1>(a, T, vcur, ic_s); break;
            case 2: batch_csr_rows<2>(a, T, vcur, ic_s); break;
            case 4: batch_csr_rows<4>(a, T, vcur, ic_s); break;
            case 8: batch_csr_rows<8>(a, T, vcur, ic_s); break;
            case 16: batch_csr_rows<16>(a, T, vcur, ic_s); break;
            default: batch_csr_rows<32>(a, T, vcur, ic_s); break;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x >= T.rows) return;
    const int64_t i = T.row0 + threadIdx.x;
    const Cell cell = load_cell(c.S, vcur, i);
    float iapp = pulse_current(c.pulses, i, t);
    if (c.iapp != nullptr) iapp += c.iapp[i];
    const CellNext o = cell_step(c.P, cell, ic_s[threadIdx.x], iapp);
    finish_cell(c, t, vnext, i, o);
}

// ---- persistent form: many steps of every network in one cooperative launch -------------
// The host cuts every network into pieces of at most 256 rows (one piece for a network
// whose work fits a CTA's share of a step, several for the large ones) and deals the
// pieces out to CTAs that are all resident at once.  Each CTA walks its pieces once per
// step.  Before reading network b's V_dend(t) it waits (bounded) until every piece of b
// has finished step t - 1: each piece adds 1 to b's arrival counter when its rows' states
// and V_dend(t + 1) are written, so b is ready for step k of the launch once its counter
// holds k x (pieces of b).  No CTA ever waits on a later step than its own, so the CTA
// with the oldest step always progresses: the launch cannot deadlock, and no grid-wide
// barrier is needed.  The pair loop, the CSR row sums and the cell update are those of
// the per-step kernel (the same lanes per row and rows per warp give the same sums), so
// the states equal those of the per-step launches bit for bit.
struct PersistItem {
    int32_t kind;     // TILE_DENSE or TILE_CSR
    int32_t net;      // network (index of its arrival counter)
    int32_t seg, n, n_pad;
    int32_t row0;     // first row (padded cell index)
    int32_t rows;     // 1..256
    int32_t pieces;   // pieces of this network (arrivals per step)
    int32_t sw;       // CSR: lanes per row
    int32_t mode;     // CSR: TileMode bits
    float g;
};

struct BatchPersistArgs {
    StepCommon c;              // par = -1; the launch runs steps *t_dev .. *t_dev + n_steps - 1
    const PersistItem *items;  // every CTA's pieces, CTA after CTA
    const int32_t *cta_off;    // [gridDim.x + 1] first piece of each CTA
    const int32_t *row_ptr;
    const uint16_t *col16;
    const float *w;
    uint32_t *cnt;             // arrival counter per network (zeroed before the launch)
    uint32_t *abort_flag;      // set by a CTA whose wait gave up (zeroed before the launch)
    uint64_t timeout_ns;
    int32_t n_steps;
    int32_t vbuf;              // floats of the staged V_dend buffer (>= n_pad of staged networks)
    int32_t kahan;
    int64_t debug_delay_ns;    // test hook: CTA 0 sleeps this long before its first piece
};

// Bounded wait until *cnt has reached target (mod 2^32), by one thread.  On timeout sets
// the timeout status bit and the abort word; returns false on timeout or abort.
__device__ __forceinline__ bool wait_arrivals(const uint32_t *cnt, uint32_t target, uint32_t *abort_flag,
                                              uint64_t timeout_ns, uint32_t *status) {
    if (arrivals_reached(ld_acquire_gpu(cnt), target)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (arrivals_reached(ld_acquire_gpu(cnt), target)) return true;
        if ((it & 63u) == 0u) {
            if (ld_acquire_gpu(abort_flag) != 0u) return false;
            if (globaltimer_ns() - t0 > timeout_ns || it > (1u << 30)) {
                atomicOr(status, (uint32_t)ST_TIMEOUT);
                atomicExch(abort_flag, 1u);
                return false;
            }
        }
    }
}

// Rows [row0, row0 + rows) of a CSR piece with 16-bit local columns: SW lanes per row,
// row voltages from vrow(local row), neighbour voltages from vj.
template <int SW, bool HAS_W, class VR, class VJ>
__device__ __forceinline__ void persist_csr_rows(const BatchPersistArgs &a, const PersistItem &P, VR vrow, VJ vj,
                                                 float *ic_s) {
    const int sub = threadIdx.x / SW, li = threadIdx.x % SW, nsub = blockDim.x / SW;
    for (int rr = sub; rr - sub < P.rows; rr += nsub) {   // the same trip count in every lane
        float acc = 0.0f;
        if (rr < P.rows) {
            const int i = P.row0 + rr;
            const int e0 = a.row_ptr[i], e1 = a.row_ptr[i + 1];
            if (e1 > e0) acc = csr_row_sum16<SW, HAS_W, false>(a.col16, a.w, e0, e1, vrow(i - P.seg), li, vj);
        }
#pragma unroll
        for (int off = SW / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (li == 0 && rr < P.rows) ic_s[rr] = (HAS_W ? acc : acc * P.g) * (1.0f / GJ_SCALE);
    }
}
template <class VR, class VJ>
__device__ __forceinline__ void persist_csr_piece(const BatchPersistArgs &a, const PersistItem &P, VR vrow, VJ vj,
                                                  float *ic_s) {
#define ION_CSR_SW(SWV)                                                                    \
    if (P.mode & TILE_UNIFORM_W) persist_csr_rows<SWV, false>(a, P, vrow, vj, ic_s);       \
    else persist_csr_rows<SWV, true>(a, P, vrow, vj, ic_s);
    switch (P.sw) {
        case 1: ION_CSR_SW(1) break;
        case 2: ION_CSR_SW(2) break;
        case 4: ION_CSR_SW(4) break;
        case 8: ION_CSR_SW(8) break;
        case 16: ION_CSR_SW(16) break;
        default: ION_CSR_SW(32) break;
    }
#undef ION_CSR_SW
}

struct VRowSmem {
    const float *v;
    __device__ __forceinline__ float operator()(int j) const { return v[j]; }
};
struct VRowCG {
    const float *v;
    __device__ __forceinline__ float operator()(int j) const { return __ldcg(v + j); }
};

// 256 threads: 8 warps; dense pieces run 8 x R rows at a time.
template <int R>
__global__ void __launch_bounds__(256, 4) batch_persist_kernel(const BatchPersistArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ float red_s[32], red_c[32];
    __shared__ float U_sh;
    __shared__ float ic_s[256];
    __shared__ int ok_sh;
    float *vb = reinterpret_cast<float *>(smem_raw);   // the piece's network's V_dend(t)
    float *part = vb + a.vbuf;                          // 8 R row partials
    const StepCommon &c = a.c;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int it0 = a.cta_off[blockIdx.x], it1 = a.cta_off[blockIdx.x + 1];
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int64_t t0 = *c.t_dev;
    uint32_t phase = 0;
    if (a.debug_delay_ns > 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        const uint64_t d0 = globaltimer_ns();
        while (globaltimer_ns() - d0 < (uint64_t)a.debug_delay_ns) __nanosleep(1000);
    }
    for (int k = 0; k < a.n_steps; ++k) {
        const int64_t t = t0 + k;
        const float *vcur = vd_slot(c.S, t);
        float *vnext = vd_slot(c.S, t + 1);
        for (int it = it0; it < it1; ++it) {
            const PersistItem P = a.items[it];
            const bool staged = P.kind == TILE_DENSE || (P.mode & TILE_STAGE_V);
            if (threadIdx.x == 0) {
                // network P.net finished step t - 1 (the launch's own earlier steps only)
                int ok = k == 0 || wait_arrivals(a.cnt + P.net, (uint32_t)k * (uint32_t)P.pieces, a.abort_flag,
                                                 a.timeout_ns, c.status);
                if (ok && staged) {
                    // the acquire above (or stream order) made the writes visible to this
                    // thread; order them before the bulk copy's async-proxy reads
                    asm volatile("fence.proxy.async;" ::: "memory");
                    mbar_expect_tx(&bar, (uint32_t)P.n_pad * 4u);
                    bulk_g2s(vb, vcur + P.seg, (uint32_t)P.n_pad * 4u, &bar);
                }
                ok_sh = ok;
            }
            __syncthreads();
            if (!ok_sh) return;
            if (staged) {
                const bool landed = mbar_wait_bounded(&bar, phase & 1u);
                phase++;
                if (__syncthreads_or(!landed)) {
                    if (threadIdx.x == 0) {
                        atomicOr(c.status, (uint32_t)ST_TIMEOUT);
                        atomicExch(a.abort_flag, 1u);
                        (void)mbar_wait_bounded(&bar, (phase - 1u) & 1u);
                    }
                    return;
                }
            }
            if (P.kind == TILE_DENSE) {
                const DenseSmem sm{vb, P.n_pad, 1, part};
                const float m_shift = vb[0];
                for (int sub = 0; sub < P.rows; sub += 8 * R) {
                    const int local0 = P.row0 - P.seg + sub;
                    const int srows = min(8 * R, P.rows - sub);
                    float ui[R];
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        ui[r] = (warp * R + r < srows) ? (vb[local0 + warp * R + r] - m_shift) * GJ_SCALE : 0.0f;
                    uint32_t uses[2] = {0u, 0u};
                    float tot[R], Us, Uc;
                    (void)gj_pass<R, 1>(sm, nullptr, P.n, P.n_pad, nullptr, uses, m_shift, ui, 0, lane, a.kahan, tot,
                                        Us, Uc);
                    const float U = gj_reduce<R, 1>(sm, tot, Us, Uc, warp, 0, lane, red_s, red_c, &U_sh);
                    if ((int)threadIdx.x < srows)
                        ic_s[sub + threadIdx.x] = row_current<1>(sm, threadIdx.x,
                                                                 (vb[local0 + threadIdx.x] - m_shift) * GJ_SCALE,
                                                                 P.n, U, P.g);
                    __syncthreads();   // part[] is rewritten by the next row block
                }
            } else if (P.mode & TILE_STAGE_V) {
                persist_csr_piece(a, P, VRowSmem{vb}, VjShared{vb}, ic_s);
            } else {
                persist_csr_piece(a, P, VRowCG{vcur + P.seg}, VjGlobalCG{vcur + P.seg}, ic_s);
            }
            __syncthreads();
            // the explicit-Euler update of the piece's rows, one thread per cell (a thread
            // reads its cell's step-t words before writing any of them)
            for (int rr = threadIdx.x; rr < P.rows; rr += blockDim.x) {
                const int64_t i = P.row0 + rr;
                const float vd = staged ? vb[i - P.seg] : __ldcg(vcur + i);
                float iapp = pulse_current(c.pulses, i, t);
                if (c.iapp != nullptr) iapp += c.iapp[i];
                const CellNext o = cell_step(c.P, load_cell(c.S, vcur, i, vd), ic_s[rr], iapp);
                finish_cell(c, t, vnext, i, o);
            }
            // every thread's reads of vb come before the next piece's bulk refill of it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            // the CTA's writes (ordered before the barrier above) precede the arrival
            if (threadIdx.x == 0) red_release_gpu_add(a.cnt + P.net, 1u);
        }
    }
}

// gather / scatter between the user's numbering (consecutive cells) and the segments
__global__ void batch_gather_kernel(const float *state, int64_t stride, const int32_t *map, int64_t n_user,
                                    int32_t vd_slot_field, float *out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_user) return;
    const int64_t src = map[j];
    for (int f = 0; f < NF; ++f) {
        const int slot = (f == 0) ? vd_slot_field : f;
        out[(int64_t)f * n_user + j] = state[(int64_t)slot * stride + src];
    }
}
__global__ void batch_scatter_kernel(float *state, int64_t stride, const int32_t *map, int64_t n_user,
                                     int32_t vd_slot_field, const float *in) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_user) return;
    const int64_t dst = map[j];
    for (int f = 0; f < NF; ++f) {
        const int slot = (f == 0) ? vd_slot_field : f;
        state[(int64_t)slot * stride + dst] = in[(int64_t)f * n_user + j];
    }
}

}  // namespace ion

using namespace ion;

// ---- host side -------------------------------------------------------------------------
struct BatchNet {
    int32_t kind, n, n_pad, seg;
    float g;          // dense: pair weight; CSR with uniform weights: every edge weight
    int64_t e0, nnz;  // CSR edges in the global arrays
    int sw;
    bool uniform = false;   // CSR: every weight bitwise equal (g)
    bool c16 = false;       // CSR: 16-bit network-local columns in col16
};

struct BatchExt {
    std::vector<BatchNet> nets;
    // persistent form (ION_FLAG_PERSISTENT): pieces dealt out to the CTAs of one
    // cooperative launch, per-network arrival counters + the abort word, and the graph of
    // one launch (counter reset, kernel, step-counter advance) for the last step count
    bool persistent = false;
    PersistItem *d_items = nullptr;
    int32_t *d_cta_off = nullptr;
    uint32_t *d_pcnt = nullptr;     // n_nets counters, then the abort word
    int p_grid = 0, p_vbuf = 256, p_pieces = 0;
    cudaGraphExec_t p_graph = nullptr;
    int64_t p_graph_steps = 0;
    bool p_graph_refused = false;
    std::vector<int32_t> h_map;     // user cell -> padded cell
    BatchTile *d_tiles = nullptr;
    int n_tiles = 0;
    int R = 2;                      // dense rows per warp (rows per dense tile = 8 R)
    int csr_rows = 128;             // rows per CSR tile
    int sw_scale = 0;               // 0: lanes per row from the degree; +-1: twice / half that
    int max_dense_pad = 256;
    float *d_tmp = nullptr;         // 19 x n_user staging for state I/O
};

static BatchExt *ext_of(ion_sim *s) { return static_cast<BatchExt *>(s->ext); }

static int csr_sw_for(double deg, int scale) {
    int sw, rows;
    ion_choose_csr_shape(deg, &sw, &rows);
    if (scale > 0 && sw < 32) sw *= 2;
    if (scale < 0 && sw > 1) sw /= 2;
    return sw;
}

// Build (or rebuild) the tile list for the current shape parameters.
static ion_status batch_plan(ion_sim *s) {
    BatchExt *X = ext_of(s);
    std::vector<BatchTile> tiles;
    std::vector<double> cost;
    const int drows = 8 * X->R;
    for (const BatchNet &b : X->nets) {
        if (b.kind == ION_DENSE_UNIFORM) {
            for (int r = 0; r < b.n; r += drows) {
                BatchTile T{TILE_DENSE, b.seg, b.n, b.n_pad, b.seg + r, std::min(drows, b.n - r), 0, b.g, 0};
                tiles.push_back(T);
                cost.push_back((double)T.rows * b.n_pad);
            }
        } else {
            const double deg = b.n > 0 ? (double)b.nnz / b.n : 0.0;
            int mode = (b.uniform ? TILE_UNIFORM_W : 0) | (b.c16 ? TILE_C16 : 0);
            if (b.c16 && b.n_pad <= X->max_dense_pad) mode |= TILE_STAGE_V;   // fits the launch's shared memory
            for (int r = 0; r < b.n; r += X->csr_rows) {
                BatchTile T{TILE_CSR, b.seg, b.n, b.n_pad, b.seg + r, std::min(X->csr_rows, b.n - r),
                            csr_sw_for(deg, X->sw_scale), b.uniform ? b.g : 0.0f, mode};
                tiles.push_back(T);
                cost.push_back(3.0 * T.rows * deg + 60.0 * T.rows);
            }
        }
    }
    std::vector<int> order(tiles.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<BatchTile> sorted(tiles.size());
    for (size_t k = 0; k < order.size(); ++k) sorted[k] = tiles[order[k]];
    cudaError_t e = cudaStreamSynchronize(s->st);
    ion_drop_graphs(s);   // the captured steps hold the old tile list
    if (e == cudaSuccess && X->d_tiles) e = cudaFree(X->d_tiles);
    X->d_tiles = nullptr;   // until a new list is in place, stepping is refused
    X->n_tiles = 0;
    if (e == cudaSuccess) e = ion_alloc(&X->d_tiles, std::max<size_t>(1, sorted.size()) * sizeof(BatchTile));
    if (e == cudaSuccess)
        e = cudaMemcpy(X->d_tiles, sorted.data(), sorted.size() * sizeof(BatchTile), cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return ion_fail(s, e == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA, "batch plan: %s", cudaGetErrorString(e));
    X->n_tiles = (int)sorted.size();
    return ION_OK;
}

// dynamic shared memory of the per-step kernel: a network's V_dend and the dense row partials
// (staging the tile's cell words here as well measured slower: fewer CTAs per SM)
static size_t batch_smem(const BatchExt *X) { return (size_t)X->max_dense_pad * 4 + 8 * X->R * 4; }

template <int R>
static cudaError_t batch_launch_R(const BatchArgs &a, int tiles, size_t smem, cudaStream_t st, bool prepare) {
    if (prepare)
        return cudaFuncSetAttribute(batch_step_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch_k(batch_step_kernel<R>, dim3(tiles), dim3(256), smem, st, a.c.pdl != 0, a);
}
static cudaError_t batch_launch(const BatchArgs &a, int R, int tiles, size_t smem, cudaStream_t st, bool prepare) {
    switch (R) {
        case 1: return batch_launch_R<1>(a, tiles, smem, st, prepare);
        case 2: return batch_launch_R<2>(a, tiles, smem, st, prepare);
        case 4: return batch_launch_R<4>(a, tiles, smem, st, prepare);
        case 8: return batch_launch_R<8>(a, tiles, smem, st, prepare);
        default: return cudaErrorInvalidValue;
    }
}

static cudaError_t batch_step(ion_sim *s, int k_off, const float *iapp) {
    BatchExt *X = ext_of(s);
    if (X->d_tiles == nullptr) return cudaErrorInvalidResourceHandle;   // no tile list: a failed re-plan
    BatchArgs a{};
    a.c = ion_step_common(s, k_off, iapp);
    a.tiles = X->d_tiles;
    a.row_ptr = s->d_rowptr;
    a.col = s->d_col;
    a.col16 = s->d_col16;
    a.w = s->d_w;
    a.kahan = 1;
    s->launches++;
    if (X->n_tiles == 0) return cudaSuccess;
    return batch_launch(a, X->R, X->n_tiles, batch_smem(X), s->st, false);
}

// ---- persistent form: planning and launch ----------------------------------------------
template <int R>
static cudaError_t persist_kernel_attr(size_t smem, int *per_sm) {
    cudaError_t e = cudaFuncSetAttribute(batch_persist_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_persist_kernel<R>, 256, smem);
    return e;
}
static cudaError_t persist_attr(int R, size_t smem, int *per_sm) {
    switch (R) {
        case 1: return persist_kernel_attr<1>(smem, per_sm);
        case 2: return persist_kernel_attr<2>(smem, per_sm);
        case 4: return persist_kernel_attr<4>(smem, per_sm);
        default: return cudaErrorInvalidValue;
    }
}
static const void *persist_fn(int R) {
    switch (R) {
        case 1: return (const void *)batch_persist_kernel<1>;
        case 2: return (const void *)batch_persist_kernel<2>;
        default: return (const void *)batch_persist_kernel<4>;
    }
}
static size_t persist_smem(const BatchExt *X) { return (size_t)X->p_vbuf * 4 + 8 * X->R * 4; }

// Cut the networks into pieces and deal them out to the CTAs of one resident grid.
// Work per row: a dense row costs its network's padded width in pair evaluations (plus a
// constant for its update), a CSR row 3 units per edge and 60 for its update; a piece
// also pays its staging.  A network becomes several pieces when its work exceeds a CTA's
// share of the total (and pieces hold at most 256 rows); pieces go largest first to the
// least loaded CTA.  Each CTA handles the pieces of networks split over several CTAs
// first, so that their arrivals come early in every step.
static ion_status batch_persist_plan(ion_sim *s) {
    BatchExt *X = ext_of(s);
    if (X->R != 1 && X->R != 2 && X->R != 4) X->R = 2;
    X->p_vbuf = X->max_dense_pad;
    int per_sm = 0;
    cudaError_t e = persist_attr(X->R, persist_smem(X), &per_sm);
    if (e != cudaSuccess || per_sm < 1)
        return ion_fail(s, ION_ERR_UNSUPPORTED, "persistent batch: no resident CTA (%s)", cudaGetErrorString(e));
    const int grid = per_sm * s->sms;
    struct Net { double per_row, fixed; int rows_align; };
    std::vector<Net> nc(X->nets.size());
    double total = 0.0;
    for (size_t b = 0; b < X->nets.size(); ++b) {
        const BatchNet &x = X->nets[b];
        if (x.kind == ION_DENSE_UNIFORM) nc[b] = {(double)x.n_pad + 64.0, 2048.0 + x.n_pad, 8 * X->R};
        else nc[b] = {3.0 * (x.n > 0 ? (double)x.nnz / x.n : 0.0) + 60.0, 2048.0 + 0.5 * x.n_pad, 32};
        total += nc[b].per_row * x.n + nc[b].fixed;
    }
    const double share = total / grid;
    struct Piece { PersistItem it; double cost; };
    std::vector<Piece> pieces;
    for (size_t b = 0; b < X->nets.size(); ++b) {
        const BatchNet &x = X->nets[b];
        const double cost = nc[b].per_row * x.n;
        int k = std::max((x.n + 255) / 256, (int)std::ceil(cost / (0.8 * share)));
        k = std::max(1, std::min(k, x.n));
        int rows = (x.n + k - 1) / k;
        const int al = nc[b].rows_align;
        rows = std::min(256, (rows + al - 1) / al * al);
        k = (x.n + rows - 1) / rows;
        for (int r = 0; r < x.n; r += rows) {
            PersistItem it{};
            it.kind = x.kind == ION_DENSE_UNIFORM ? TILE_DENSE : TILE_CSR;
            it.net = (int32_t)b;
            it.seg = x.seg;
            it.n = x.n;
            it.n_pad = x.n_pad;
            it.row0 = x.seg + r;
            it.rows = std::min(rows, x.n - r);
            it.pieces = k;
            it.g = x.g;
            if (x.kind != ION_DENSE_UNIFORM) {
                it.sw = x.sw;
                it.mode = (x.uniform ? TILE_UNIFORM_W : 0) | (x.c16 ? TILE_C16 : 0);
                if (x.c16 && x.n_pad <= X->p_vbuf) it.mode |= TILE_STAGE_V;
            }
            pieces.push_back({it, nc[b].per_row * it.rows + nc[b].fixed});
        }
    }
    std::vector<int> order(pieces.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pieces[a].cost > pieces[b].cost; });
    std::vector<double> load((size_t)grid, 0.0);
    std::vector<std::vector<int>> own((size_t)grid);
    for (int q : order) {
        const size_t c = (size_t)(std::min_element(load.begin(), load.end()) - load.begin());
        load[c] += pieces[q].cost;
        own[c].push_back(q);
    }
    std::vector<PersistItem> items;
    std::vector<int32_t> off((size_t)grid + 1, 0);
    for (int c = 0; c < grid; ++c) {
        std::vector<int> &L = own[(size_t)c];
        std::stable_sort(L.begin(), L.end(), [&](int a, int b) {
            const PersistItem &A = pieces[a].it, &B = pieces[b].it;
            if ((A.pieces > 1) != (B.pieces > 1)) return A.pieces > 1;
            return A.row0 < B.row0;
        });
        for (int q : L) items.push_back(pieces[q].it);
        off[(size_t)c + 1] = (int32_t)items.size();
    }
    e = cudaStreamSynchronize(s->st);
    if (X->p_graph) {
        cudaGraphExecDestroy(X->p_graph);
        X->p_graph = nullptr;
        X->p_graph_steps = 0;
    }
    cudaFree(X->d_items);
    cudaFree(X->d_cta_off);
    X->d_items = nullptr;
    X->d_cta_off = nullptr;
    X->p_grid = 0;
    if (e == cudaSuccess) e = ion_alloc(&X->d_items, std::max<size_t>(1, items.size()) * sizeof(PersistItem));
    if (e == cudaSuccess) e = ion_alloc(&X->d_cta_off, off.size() * sizeof(int32_t));
    if (e == cudaSuccess && !X->d_pcnt) e = ion_alloc(&X->d_pcnt, (X->nets.size() + 1) * sizeof(uint32_t));
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpy(X->d_items, items.data(), items.size() * sizeof(PersistItem), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(X->d_cta_off, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return ion_fail(s, e == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA, "persistent batch plan: %s",
                        cudaGetErrorString(e));
    X->p_grid = grid;
    X->p_pieces = (int)items.size();
    return ION_OK;
}

// One launch of n_steps steps: counters and abort word cleared, the cooperative kernel,
// then the device step counter advanced.
static cudaError_t persist_enqueue(ion_sim *s, int n_steps, bool capture) {
    BatchExt *X = ext_of(s);
    BatchPersistArgs a{};
    a.c = ion_step_common(s, 0, nullptr);
    a.c.par = -1;   // many steps per launch: the slots follow the device counter
    a.items = X->d_items;
    a.cta_off = X->d_cta_off;
    a.row_ptr = s->d_rowptr;
    a.col16 = s->d_col16;
    a.w = s->d_w;
    a.cnt = X->d_pcnt;
    a.abort_flag = X->d_pcnt + X->nets.size();
    a.timeout_ns = s->barrier_timeout_ns;
    a.n_steps = n_steps;
    a.vbuf = X->p_vbuf;
    a.kahan = 1;
    a.debug_delay_ns = s->debug_delay_ns;
    cudaError_t e = cudaMemsetAsync(X->d_pcnt, 0, (X->nets.size() + 1) * sizeof(uint32_t), s->st);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    if (capture) {
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(X->p_grid);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = persist_smem(X);
        cfg.stream = s->st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelExC(&cfg, persist_fn(X->R), args);
    } else {
        e = cudaLaunchCooperativeKernel(persist_fn(X->R), dim3(X->p_grid), dim3(256), args, persist_smem(X), s->st);
    }
    if (e != cudaSuccess) return e;
    return launch_advance(s->d_t, n_steps, s->st);
}

// The captured launch holds the pulse table and trace ring of its capture: dropped with
// the per-step graphs whenever those change.
static void batch_persist_drop(ion_sim *s) {
    BatchExt *X = ext_of(s);
    if (X && X->p_graph) {
        cudaGraphExecDestroy(X->p_graph);
        X->p_graph = nullptr;
        X->p_graph_steps = 0;
    }
}

// ion_step of a persistent batch: one graph replay (or, where a capture is refused, one
// direct cooperative launch) per 2^22 steps.
static ion_status batch_persist_run(ion_sim *s, int64_t n_steps, const float *iapp) {
    (void)iapp;
    BatchExt *X = ext_of(s);
    if (X->d_items == nullptr || X->p_grid == 0) return ion_fail(s, ION_ERR_CUDA, "persistent batch: no plan");
    int64_t done = 0;
    while (done < n_steps) {
        const int chunk = (int)std::min<int64_t>(n_steps - done, 1 << 22);
        cudaError_t e = cudaSuccess;
        if (!X->p_graph_refused && X->p_graph_steps != chunk) {
            if (X->p_graph) cudaGraphExecDestroy(X->p_graph);
            X->p_graph = nullptr;
            X->p_graph_steps = 0;
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t e1 = persist_enqueue(s, chunk, true);
                const cudaError_t e2 = cudaStreamEndCapture(s->st, &g);
                e = e1 != cudaSuccess ? e1 : e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&X->p_graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e == cudaSuccess) {
                X->p_graph_steps = chunk;
            } else {   // no cooperative launches in graphs here: launch directly from now on
                (void)cudaGetLastError();
                X->p_graph = nullptr;
                X->p_graph_refused = true;
            }
        }
        if (X->p_graph != nullptr && X->p_graph_steps == chunk) e = cudaGraphLaunch(X->p_graph, s->st);
        else e = persist_enqueue(s, chunk, false);
        s->launches += 2;
        if (e != cudaSuccess) return ion_fail(s, ION_ERR_CUDA, "persistent batch launch: %s", cudaGetErrorString(e));
        done += chunk;
    }
    return ION_OK;
}

static ion_status batch_prepare(ion_sim *s) {
    BatchExt *X = ext_of(s);
    cudaError_t e = batch_launch(BatchArgs{}, X->R, 0, batch_smem(X), s->st, true);
    if (e != cudaSuccess) return ion_fail(s, ION_ERR_CUDA, "batch setup: %s", cudaGetErrorString(e));
    return ION_OK;
}

// state I/O in the user's numbering
ion_status ion_batch_read(ion_sim *s, int32_t field, float *out) {
    BatchExt *X = ext_of(s);
    const int64_t nu = (int64_t)X->h_map.size();
    const int vd = (s->t & 1) ? 19 : 0;
    batch_gather_kernel<<<(unsigned)((nu + 255) / 256), 256, 0, s->st>>>(s->d_state, s->stride, s->d_map, nu, vd,
                                                                        X->d_tmp);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e == cudaSuccess) {
        if (field == ION_FIELD_ALL)
            e = cudaMemcpy(out, X->d_tmp, (size_t)NF * nu * sizeof(float), cudaMemcpyDeviceToHost);
        else
            e = cudaMemcpy(out, X->d_tmp + (int64_t)field * nu, (size_t)nu * sizeof(float), cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return ion_fail(s, ION_ERR_CUDA, "batch read: %s", cudaGetErrorString(e));
    return ION_OK;
}

ion_status ion_batch_write(ion_sim *s, int32_t field, const float *in) {
    BatchExt *X = ext_of(s);
    const int64_t nu = (int64_t)X->h_map.size();
    const int vd = (s->t & 1) ? 19 : 0;
    cudaError_t e = cudaSuccess;
    if (field != ION_FIELD_ALL) {   // read-modify-write of the one field through the staging buffer
        batch_gather_kernel<<<(unsigned)((nu + 255) / 256), 256, 0, s->st>>>(s->d_state, s->stride, s->d_map, nu, vd,
                                                                            X->d_tmp);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
        if (e == cudaSuccess)
            e = cudaMemcpy(X->d_tmp + (int64_t)field * nu, in, (size_t)nu * sizeof(float), cudaMemcpyHostToDevice);
    } else {
        e = cudaMemcpy(X->d_tmp, in, (size_t)NF * nu * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        batch_scatter_kernel<<<(unsigned)((nu + 255) / 256), 256, 0, s->st>>>(s->d_state, s->stride, s->d_map, nu, vd,
                                                                             X->d_tmp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return ion_fail(s, ION_ERR_CUDA, "batch write: %s", cudaGetErrorString(e));
    return ION_OK;
}

int32_t ion_batch_map_cell(ion_sim *s, int64_t user_cell) {
    BatchExt *X = ext_of(s);
    if (user_cell < 0 || user_cell >= (int64_t)X->h_map.size()) return -1;
    return X->h_map[(size_t)user_cell];
}

static void batch_free(ion_sim *s) {
    BatchExt *X = ext_of(s);
    if (!X) return;
    s->drop_hook = nullptr;
    if (X->p_graph) cudaGraphExecDestroy(X->p_graph);
    cudaFree(X->d_items);
    cudaFree(X->d_cta_off);
    cudaFree(X->d_pcnt);
    cudaFree(X->d_tiles);
    cudaFree(X->d_tmp);
    cudaFree(s->d_map);
    s->d_map = nullptr;
    delete X;
    s->ext = nullptr;
}

extern "C" ion_status ion_create_batch(int32_t n_nets, const ion_net *nets, const ion_conn *conns,
                                       const ion_params *params, const float *init_state, ion_sim **out) {
    if (!out) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create_batch: NULL out");
    *out = nullptr;
    if (n_nets < 1 || !nets || !conns || !params)
        return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create_batch: bad arguments");
    if (params->flags & (ION_FLAG_SURROGATE | ION_FLAG_SPLIT | ION_FLAG_SGJ))
        return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "ion_create_batch: flags not supported for batches");
    if ((params->flags & ION_FLAG_PERSISTENT) && (params->flags & ION_FLAG_CSR_AS_GIVEN))
        return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "ion_create_batch: a persistent batch needs the compact CSR layout");
    if (params->cell_params)
        return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "ion_create_batch: per-cell constants not supported for batches");
    // validate and lay out
    std::vector<BatchNet> bn((size_t)n_nets);
    int64_t seg = 0, n_user = 0, nnz_total = 0;
    int max_pad = 256;
    for (int b = 0; b < n_nets; ++b) {
        const ion_net &N = nets[b];
        if (N.n_cells < 1 || (N.kind != ION_DENSE_UNIFORM && N.kind != ION_CSR && N.kind != ION_NO_GJ))
            return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create_batch: network %d: bad size or kind", b);
        if (N.kind == ION_DENSE_UNIFORM && N.n_cells > TJ)
            return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "ion_create_batch: dense network %d has %d > %d cells", b,
                            N.n_cells, TJ);
        if (N.kind == ION_DENSE_UNIFORM && !std::isfinite(conns[b].g_c))
            return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create_batch: network %d: g_c not finite", b);
        if (N.kind == ION_CSR) {
            if (conns[b].mem != ION_HOST)
                return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "ion_create_batch: network %d: CSR must be host memory", b);
            ion_status st = ion_validate_csr(N.n_cells, &conns[b]);
            if (st != ION_OK) return st;
        }
        BatchNet &x = bn[(size_t)b];
        x.kind = N.kind;
        x.n = N.n_cells;
        x.n_pad = (N.n_cells + PAD_J - 1) / PAD_J * PAD_J;
        x.seg = (int32_t)seg;
        x.g = N.kind == ION_DENSE_UNIFORM ? conns[b].g_c : 0.0f;
        x.e0 = nnz_total;
        x.nnz = N.kind == ION_CSR ? conns[b].nnz : 0;
        if (N.kind == ION_CSR && !(params->flags & ION_FLAG_CSR_AS_GIVEN)) {
            // compact layout: 16-bit local columns; one scalar when every weight is bitwise equal
            x.c16 = N.n_cells <= 65536;
            const ion_conn &C = conns[b];
            x.uniform = true;
            x.g = C.g_c;
            if (C.weight && x.nnz > 0) {
                uint32_t b0, be;
                std::memcpy(&b0, C.weight, sizeof b0);
                for (int64_t q = 1; q < x.nnz && x.uniform; ++q) {
                    std::memcpy(&be, C.weight + q, sizeof be);
                    x.uniform = be == b0;
                }
                x.g = C.weight[0];
            }
        }
        if (N.kind == ION_DENSE_UNIFORM || (x.c16 && x.n_pad <= TJ)) max_pad = std::max(max_pad, x.n_pad);
        seg += x.n_pad;
        n_user += x.n;
        nnz_total += x.nnz;
        if (seg >= (1 << 30) || nnz_total >= INT32_MAX)
            return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create_batch: batch too large");
    }
    // create an empty single-network handle of the padded size, then turn it into a batch
    ion_net whole{(int32_t)seg, ION_NO_GJ};
    ion_params p = *params;
    p.flags &= ~(uint32_t)ION_FLAG_PERSISTENT;
    ion_sim *s = nullptr;
    ion_status st = ion_create(&whole, nullptr, &p, nullptr, &s);
    if (st != ION_OK) return st;
    auto fail = [&](ion_status code) {
        ion_destroy(s);
        return code;
    };
    BatchExt *X = new BatchExt();
    s->ext = X;
    s->extra_free = batch_free;
    X->nets = bn;
    X->max_dense_pad = max_pad;
    X->h_map.resize((size_t)n_user);
    {
        int64_t u = 0;
        for (const BatchNet &x : bn)
            for (int i = 0; i < x.n; ++i) X->h_map[(size_t)u++] = x.seg + i;
    }
    const ion_tune *tu = (const ion_tune *)params->tune;
    if (tu && tu->dense_rows_per_warp > 0) X->R = tu->dense_rows_per_warp;
    if (tu && tu->csr_rows_per_cta > 0) X->csr_rows = tu->csr_rows_per_cta;
    if (tu && tu->csr_lanes_scale != 0) X->sw_scale = tu->csr_lanes_scale > 0 ? 1 : -1;
    if ((X->R != 1 && X->R != 2 && X->R != 4 && X->R != 8) || X->csr_rows < 1 || X->csr_rows > 256)
        return fail(ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create_batch: bad tile shape override"));
    // global CSR over the padded index space
    std::vector<int32_t> rp((size_t)seg + 1, 0), col((size_t)std::max<int64_t>(nnz_total, 1));
    std::vector<float> w((size_t)std::max<int64_t>(nnz_total, 1));
    std::vector<uint16_t> col16((size_t)(nnz_total + 8), 0);   // padded to whole 16-byte groups
    bool any16 = false;
    for (int b = 0; b < n_nets; ++b) {
        const BatchNet &x = bn[(size_t)b];
        if (x.kind != ION_CSR) continue;
        const ion_conn &C = conns[b];
        any16 = any16 || x.c16;
        for (int i = 0; i < x.n; ++i) rp[(size_t)x.seg + i + 1] = C.row_ptr[i + 1] - C.row_ptr[i];
        for (int64_t e = 0; e < x.nnz; ++e) {
            col[(size_t)(x.e0 + e)] = x.seg + C.col_idx[e];
            w[(size_t)(x.e0 + e)] = C.weight ? C.weight[e] : C.g_c;
            if (x.c16) col16[(size_t)(x.e0 + e)] = (uint16_t)C.col_idx[e];
        }
    }
    for (size_t i = 0; i < (size_t)seg; ++i) rp[i + 1] += rp[i];
    // the per-row counts above were placed in network order, so the prefix sum lines the
    // edges up with x.e0 (segments are laid out in network order)
    s->own_csr = true;   // before the allocations, so that a partial failure frees them
    cudaError_t e = ion_alloc(&s->d_rowptr, rp.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = ion_alloc(&s->d_col, col.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = ion_alloc(&s->d_w, w.size() * sizeof(float));
    if (e == cudaSuccess && any16) e = ion_alloc(&s->d_col16, col16.size() * sizeof(uint16_t));
    if (e == cudaSuccess) e = ion_alloc(&s->d_map, X->h_map.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = ion_alloc(&X->d_tmp, (size_t)NF * n_user * sizeof(float));
    if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_OOM, "ion_create_batch: %s", cudaGetErrorString(e)));
    s->nnz = nnz_total;
    e = cudaMemcpy(s->d_rowptr, rp.data(), rp.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_col, col.data(), col.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_w, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && any16)
        e = cudaMemcpy(s->d_col16, col16.data(), col16.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->d_map, X->h_map.data(), X->h_map.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_CUDA, "ion_create_batch: %s", cudaGetErrorString(e)));
    for (BatchNet &x : X->nets)
        if (x.kind == ION_CSR) x.sw = csr_sw_for((double)x.nnz / x.n, 0);
    s->kind = ION_CSR;   // the generic paths see a CSR handle; stepping is overridden
    s->n_user = n_user;
    s->step_override = batch_step;
    s->prepare_hook = nullptr;
    // every V_dend padding cell holds the sentinel (the default state wrote V_0 there)
    for (const BatchNet &x : X->nets) {
        if (x.n_pad > x.n) {
            e = launch_fill(s->d_state + x.seg + x.n, PAD_VOLT, x.n_pad - x.n, s->st);
            if (e == cudaSuccess) e = launch_fill(s->d_state + 19 * s->stride + x.seg + x.n, PAD_VOLT, x.n_pad - x.n, s->st);
            if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_CUDA, "ion_create_batch: %s", cudaGetErrorString(e)));
        }
    }
    if (init_state) {
        st = ion_batch_write(s, ION_FIELD_ALL, init_state);
        if (st != ION_OK) return fail(st);
    }
    st = batch_plan(s);
    if (st == ION_OK) st = batch_prepare(s);
    if (st != ION_OK) return fail(st);
    if (params->flags & ION_FLAG_PERSISTENT) {
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device);
        if (!coop) return fail(ion_fail(nullptr, ION_ERR_UNSUPPORTED, "ion_create_batch: no cooperative launches"));
        X->persistent = true;
        s->flags |= ION_FLAG_PERSISTENT;
        st = batch_persist_plan(s);
        if (st != ION_OK) return fail(st);
        s->run_override = batch_persist_run;
        s->drop_hook = batch_persist_drop;
    }
    *out = s;
    return ION_OK;
}

// ---- autotuner ------------------------------------------------------------------------------
// Times candidate launch shapes on the handle's own network(s), `steps` time steps each
// (direct launches, CUDA events), and keeps the fastest.  The state and step count are
// saved before and restored after, so tuning does not advance the simulation.
static ion_status time_steps(ion_sim *s, int steps, float *ms) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int64_t t_save = s->t;
    cudaEventRecord(a, s->st);
    const uint32_t flags = s->flags;
    s->flags |= ION_FLAG_NO_GRAPH;
    ion_status st = ion_step(s, steps, nullptr);
    s->flags = flags;
    cudaEventRecord(b, s->st);
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    (void)t_save;
    if (st != ION_OK) return st;
    if (e != cudaSuccess) return ion_fail(s, ION_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(e));
    return ION_OK;
}

static ion_status autotune_persist_batch(ion_sim *s, int32_t steps, ion_tune *chosen);

extern "C" ion_status ion_autotune(ion_sim *s, int32_t steps, ion_tune *chosen) {
    if (!s || steps < 1) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_autotune: bad arguments");
    if (s->ext && s->run_override == batch_persist_run) return autotune_persist_batch(s, steps, chosen);
    if (s->run_override) return ion_fail(s, ION_ERR_UNSUPPORTED, "ion_autotune: persistent handles are not tuned");
    // save the state and the step counter
    float *save = nullptr;
    const size_t bytes = (size_t)20 * s->stride * sizeof(float);
    cudaError_t e = cudaStreamSynchronize(s->st);
    if (e == cudaSuccess) e = ion_alloc(&save, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(save, s->d_state, bytes, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
        cudaFree(save);
        return ion_fail(s, e == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA, "ion_autotune: %s",
                        cudaGetErrorString(e));
    }
    const int64_t t0 = s->t;
    auto restore = [&]() {
        cudaStreamSynchronize(s->st);
        cudaMemcpy(s->d_state, save, bytes, cudaMemcpyDeviceToDevice);
        cudaMemcpy(s->d_t, &t0, sizeof t0, cudaMemcpyHostToDevice);
        s->t = t0;
    };
    float best = 1e30f;
    ion_tune bt{};
    ion_status st = ION_OK;
    if (s->ext && s->step_override == batch_step) {
        BatchExt *X = ext_of(s);
        const int Rs[] = {1, 2, 4, 8};
        const int rows[] = {64, 128, 256};
        const int scales[] = {0, 1, -1};
        int bR = X->R, brows = X->csr_rows, bsc = X->sw_scale;
        for (int R : Rs)
            for (int r : rows)
                for (int sc : scales) {
                    X->R = R;
                    X->csr_rows = r;
                    X->sw_scale = sc;
                    st = batch_plan(s);
                    if (st == ION_OK) st = batch_prepare(s);
                    float ms = 0;
                    if (st == ION_OK) st = time_steps(s, steps, &ms);
                    restore();
                    if (st != ION_OK) break;
                    if (ms < best) {
                        best = ms;
                        bR = R;
                        brows = r;
                        bsc = sc;
                    }
                }
        X->R = bR;
        X->csr_rows = brows;
        X->sw_scale = bsc;
        if (st == ION_OK) st = batch_plan(s);
        if (st == ION_OK) st = batch_prepare(s);
        bt.dense_rows_per_warp = bR;
        bt.dense_warps = 8;
        bt.dense_col_splits = 1;
        bt.csr_rows_per_cta = brows;
        bt.csr_lanes_scale = bsc;     // scale of the degree-based choice: 0, +1 (x2), -1 (/2)
    } else if (s->kind == ION_DENSE_UNIFORM) {
        int R0, W0, G0;
        ion_choose_dense_shape(s->n, s->sms, &R0, &W0, &G0);
        struct Shape { int R, W, GJ; };
        std::vector<Shape> cand = {{R0, W0, G0}};
        const int Rs[] = {1, 2, 4, 6, 8};
        const int GJs[] = {1, 2, 4};
        for (int R : Rs)
            for (int GJ : GJs)
                for (int GR = 1; GR <= 32; ++GR) {
                    const int W = GR * GJ;
                    if (W * 32 > dense_max_threads(R) || W < 8) continue;
                    const long rows_cta = (long)GR * R;
                    const long grid = (s->n + rows_cta - 1) / rows_cta;
                    const long cost = ((grid + s->sms - 1) / s->sms) * (rows_cta + 4);
                    const long grid0 = (s->n + (long)(W0 / G0) * R0 - 1) / ((long)(W0 / G0) * R0);
                    const long cost0 = ((grid0 + s->sms - 1) / s->sms) * ((long)(W0 / G0) * R0 + 4);
                    if (cost <= cost0 * 11 / 10 && cand.size() < 12 && !(R == R0 && W == W0 && GJ == G0))
                        cand.push_back({R, W, GJ});
                }
        Shape bs = cand[0];
        for (const Shape &c : cand) {
            if (prepare_dense_step(c.R, c.W, c.GJ, s->n_pad) != cudaSuccess) continue;
            s->dense_R = c.R;
            s->dense_W = c.W;
            s->dense_GJ = c.GJ;
            float ms = 0;
            st = time_steps(s, steps, &ms);
            restore();
            if (st != ION_OK) break;
            if (ms < best) {
                best = ms;
                bs = c;
            }
        }
        s->dense_R = bs.R;
        s->dense_W = bs.W;
        s->dense_GJ = bs.GJ;
        prepare_dense_step(bs.R, bs.W, bs.GJ, s->n_pad);
        bt.dense_rows_per_warp = bs.R;
        bt.dense_warps = bs.W;
        bt.dense_col_splits = bs.GJ;
    } else if (s->kind == ION_DENSE_MATRIX) {
        int bR = s->dense_R;
        for (int R : {1, 2, 4}) {
            s->dense_R = R;
            float ms = 0;
            st = time_steps(s, steps, &ms);
            restore();
            if (st != ION_OK) break;
            if (ms < best) {
                best = ms;
                bR = R;
            }
        }
        s->dense_R = bR;
        bt.dense_rows_per_warp = bR;
        bt.dense_warps = 8;
        bt.dense_col_splits = 1;
    } else if (s->kind == ION_CSR) {
        const int SWs[] = {1, 2, 4, 8, 16, 32};
        const int rows[] = {32, 64, 128, 256};
        int bsw = s->csr_SW, brows = s->csr_rows, bstaged = s->csr_staged;
        int b_csw = s->csr_chunk_SW;
        const int sw0 = s->csr_SW;
        for (int staged = 0; staged <= 1 && st == ION_OK; ++staged) {
            if (staged) {
                if (ion_setup_csr_staging(s, 2) != ION_OK || s->csr_staged == 0) break;
            } else {
                s->csr_staged = 0;
            }
            const int mode = s->csr_staged;
            for (int sw : SWs) {
                if (sw * 4 < sw0 || sw > sw0 * 4) continue;   // near the degree-based choice
                for (int r : rows) {
                    if (staged && r != rows[0]) continue;     // staged: rows per CTA fixed by the SM count
                    if (staged) {
                        s->csr_chunk_SW = sw;
                        st = ion_prepare_csr_chunk(s);
                        if (st != ION_OK) break;
                    } else {
                        s->csr_SW = sw;
                        s->csr_rows = r;
                    }
                    float ms = 0;
                    st = time_steps(s, steps, &ms);
                    restore();
                    if (st != ION_OK) break;
                    if (ms < best) {
                        best = ms;
                        bstaged = mode;
                        if (staged) b_csw = sw;
                        else {
                            bsw = sw;
                            brows = r;
                        }
                    }
                }
            }
        }
        s->csr_SW = bsw;
        s->csr_rows = brows;
        s->csr_staged = bstaged;
        s->csr_chunk_SW = b_csw;
        bt.csr_lanes_per_row = bstaged ? b_csw : bsw;
        bt.csr_rows_per_cta = bstaged ? s->csr_chunk_rows : brows;
        bt.csr_staging = bstaged ? 2 : 1;
    }
    ion_drop_graphs(s);
    cudaFree(save);
    if (st != ION_OK) return st;
    if (chosen) *chosen = bt;
    return ION_OK;
}

// Persistent batches: rows per warp of the dense pieces (1, 2 or 4), each timed over
// `steps` steps of one launch, the state and step count restored after each.
static ion_status autotune_persist_batch(ion_sim *s, int32_t steps, ion_tune *chosen) {
    BatchExt *X = ext_of(s);
    float *save = nullptr;
    const size_t bytes = (size_t)20 * s->stride * sizeof(float);
    cudaError_t e = cudaStreamSynchronize(s->st);
    if (e == cudaSuccess) e = ion_alloc(&save, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(save, s->d_state, bytes, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
        cudaFree(save);
        return ion_fail(s, e == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA, "ion_autotune: %s",
                        cudaGetErrorString(e));
    }
    const int64_t t0 = s->t;
    float best = 1e30f;
    int bR = X->R;
    ion_status st = ION_OK;
    for (int R : {1, 2, 4}) {
        X->R = R;
        st = batch_persist_plan(s);
        if (st != ION_OK) break;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s->st);
        st = batch_persist_run(s, steps, nullptr);
        cudaEventRecord(b, s->st);
        float ms = 0.0f;
        e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        cudaMemcpy(s->d_state, save, bytes, cudaMemcpyDeviceToDevice);
        cudaMemcpy(s->d_t, &t0, sizeof t0, cudaMemcpyHostToDevice);
        s->t = t0;
        if (st != ION_OK) break;
        if (e != cudaSuccess) {
            st = ion_fail(s, ION_ERR_CUDA, "ion_autotune: %s", cudaGetErrorString(e));
            break;
        }
        if (ms < best) {
            best = ms;
            bR = R;
        }
    }
    X->R = bR;
    if (st == ION_OK) st = batch_persist_plan(s);
    if (st == ION_OK) st = batch_prepare(s);   // the per-step kernel (dense inputs) uses R too
    if (st == ION_OK) st = batch_plan(s);
    cudaFree(save);
    if (st != ION_OK) return st;
    if (chosen) {
        *chosen = ion_tune{};
        chosen->dense_rows_per_warp = bR;
        chosen->dense_warps = 8;
        chosen->dense_col_splits = 1;
        chosen->csr_rows_per_cta = X->csr_rows;
    }
    return ION_OK;
}
