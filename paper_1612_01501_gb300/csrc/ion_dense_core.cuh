// ion_dense_core.cuh -- the dense gap-junction pass shared by the single-network kernels
// (ion_dense.cu) and the batched kernel (ion_batch.cu): staging of V_dend tiles, the
// centred/scaled/negated tile, the packed pair loop with Kahan folds, the fixed-order
// reductions and the per-row current.  See ion_dense.cu for the arithmetic.
#pragma once
#include <cstdint>

#include "ion_async.cuh"
#include "ion_kernels.cuh"

namespace ion {

constexpr float PAD_U = 1.0e6f;   // |u| of padded columns: 2^{-PAD_U^2} is exactly 0 (matrix kernel)

struct DenseSmem {
    float *tile0;     // buffer b at tile0 + b * buf_len
    int buf_len;
    int n_tiles;
    float *part;      // [rows_cta][GJ] row sums per column split
};

__device__ __forceinline__ DenseSmem dense_smem(unsigned char *raw, int n_pad) {
    DenseSmem s;
    s.tile0 = reinterpret_cast<float *>(raw);
    s.n_tiles = (n_pad + TJ - 1) / TJ;
    s.buf_len = s.n_tiles > 1 ? TJ : n_pad;
    s.part = s.tile0 + (s.n_tiles > 1 ? 2 * TJ : n_pad);
    return s;
}

// Issue the bulk copy of tile k (thread 0 only).
__device__ __forceinline__ void issue_tile(const DenseSmem &sm, const float *src, int n_pad, int k, uint64_t *bar) {
    const int len = min(TJ, n_pad - k * TJ);
    mbar_expect_tx(&bar[k & 1], (uint32_t)len * 4u);
    bulk_g2s(sm.tile0 + (k & 1) * sm.buf_len, src + (int64_t)k * TJ, (uint32_t)len * 4u, &bar[k & 1]);
}

// One block of the pair loop: BLK float4 columns of one lane (m0, m0 + 32 GJ, ...), every
// column against the lane's R rows, summed into acc[r].  CHECK: the block may run past n4
// (the last block of a tile), so each column is tested; a full block runs without tests.
template <int R, int GJ, int BLK, bool CHECK>
__device__ __forceinline__ void gj_block(const float4 *t4, int m0, int n4, float2 negm2, float2 negs2,
                                         const float2 (&u2)[R], float2 (&acc)[R]) {
#pragma unroll 4
    for (int mm = 0; mm < BLK; ++mm) {
        const int m = m0 + mm * 32 * GJ;
        if (CHECK && m >= n4) break;
        const float4 v = t4[m];
        const float2 va = __fmul2_rn(__fadd2_rn(make_float2(v.x, v.y), negm2), negs2);
        const float2 vb = __fmul2_rn(__fadd2_rn(make_float2(v.z, v.w), negm2), negs2);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 da = __fadd2_rn(u2[r], va);
            const float2 db = __fadd2_rn(u2[r], vb);
            const float2 qa = __fmul2_rn(da, da);
            const float2 qb = __fmul2_rn(db, db);
            const float2 ea = make_float2(ex2_approx(-qa.x), ex2_approx(-qa.y));
            const float2 eb = make_float2(ex2_approx(-qb.x), ex2_approx(-qb.y));
            acc[r] = __ffma2_rn(ea, da, acc[r]);
            acc[r] = __ffma2_rn(eb, db, acc[r]);
        }
    }
}

// One pass over all columns.  If `src` is non-NULL the first two tiles must already be in
// flight (issue_tile) and the remaining ones are issued here; if NULL the single tile
// already holds V_dend (single-CTA persistent mode).  The tiles hold raw V_dend: each lane
// centres, scales and negates the four columns of a 16-byte load as it reads them,
// x_j = -(V_j - m) s, so there is no pass over the tile between its arrival and the pair
// loop.  Columns past the last real cell are skipped.  After a tile's pairs, every warp
// adds up its even share of the tile's real x_j (the linear part's sum_j u_j is not
// needed before the reduction, and an even share keeps the warps balanced).  On return
// tot[r] holds this lane's compensated column sum for row r, and (Us, Uc) this thread's
// compensated share of sum_j u_j.  bar_uses counts completed phases of each mbarrier.
// Returns false (in every thread) if a bulk copy did not land in time.
template <int R, int GJ>
__device__ __forceinline__ bool gj_pass(const DenseSmem &sm, const float *src, int n, int n_pad, uint64_t *bar,
                                        uint32_t (&bar_uses)[2], float m_shift, const float (&ui)[R], int cs,
                                        int lane, int kahan, float (&tot)[R], float &Us, float &Uc) {
    float ks[R], kc[R];
    float2 u2[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        ks[r] = kc[r] = 0.0f;
        u2[r] = make_float2(ui[r], ui[r]);
    }
    float ns = 0.0f, nc = 0.0f;   // compensated sum of x = -u over this thread's share of columns
    const float2 negm2 = make_float2(-m_shift, -m_shift);
    const float2 negs2 = make_float2(-GJ_SCALE, -GJ_SCALE);
    constexpr int BLK = 16;       // float4 loads per lane between Kahan folds
    for (int kt = 0; kt < sm.n_tiles; ++kt) {
        const int b = kt & 1;
        const int j0 = kt * TJ;
        const int len = min(TJ, n_pad - j0);
        if (src != nullptr) {
            const bool landed = mbar_wait_bounded(&bar[b], bar_uses[b] & 1u);
            bar_uses[b]++;
            if (__syncthreads_or(!landed)) return false;   // block-uniform decision
        }
        const float *tb = sm.tile0 + b * sm.buf_len;
        const float4 *t4 = reinterpret_cast<const float4 *>(tb);
        const int real = max(0, min(len, n - j0));   // real columns of this tile
        const int n4 = (real + 3) >> 2;               // float4 columns that hold any
        // The pair loop runs to a multiple of 32 float4 columns (within the padded tile),
        // so that a warp's 32 lanes are all in range or all out: no lane of a warp takes
        // the checked path while another takes the unchecked one.  The columns added are
        // sentinel padding, whose pairs contribute exactly 0.
        const int n4w = min((n4 + 31) & ~31, len >> 2);
        for (int m0 = cs * 32 + lane; m0 < n4w; m0 += 32 * GJ * BLK) {
            float2 acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = make_float2(0.0f, 0.0f);
            if (m0 + (BLK - 1) * 32 * GJ < n4w) gj_block<R, GJ, BLK, false>(t4, m0, n4w, negm2, negs2, u2, acc);
            else gj_block<R, GJ, BLK, true>(t4, m0, n4w, negm2, negs2, u2, acc);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float blk = acc[r].x + acc[r].y;
                if (kahan) kahan_add(ks[r], kc[r], blk);
                else ks[r] += blk;
            }
        }
        // this thread's share of the tile's real x_j, the same transform as above
        for (int j4 = threadIdx.x; j4 < n4; j4 += blockDim.x) {
            const float4 v = t4[j4];
            const float2 va = __fmul2_rn(__fadd2_rn(make_float2(v.x, v.y), negm2), negs2);
            const float2 vb = __fmul2_rn(__fadd2_rn(make_float2(v.z, v.w), negm2), negs2);
            const int rem = real - 4 * j4;   // real columns in this float4 (>= 1)
            float x = va.x;
            if (rem > 1) x += va.y;
            if (rem > 2) x += vb.x;
            if (rem > 3) x += vb.y;
            kahan_add(ns, nc, x);
        }
        // order this thread's generic accesses of the buffer before any later bulk refill
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (src != nullptr && kt + 2 < sm.n_tiles) {   // refilled now: every thread must be done with it
            __syncthreads();
            if (threadIdx.x == 0) issue_tile(sm, src, n_pad, kt + 2, bar);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) tot[r] = ks[r] - kc[r];
    Us = -ns;   // sum of u = -(sum of x)
    Uc = -nc;
    return true;
}

// Reduce the lane sums into part[row][split] and the block's sum_j u_j (returned).
template <int R, int GJ>
__device__ __forceinline__ float gj_reduce(const DenseSmem &sm, const float (&tot)[R], float Us, float Uc, int rg,
                                           int cs, int lane, float *red_s, float *red_c, float *U_sh) {
    const int warp = threadIdx.x >> 5, W = blockDim.x >> 5;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float v = tot[r];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) sm.part[(rg * R + r) * GJ + cs] = v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Us += __shfl_xor_sync(0xffffffffu, Us, off);
        Uc += __shfl_xor_sync(0xffffffffu, Uc, off);
    }
    if (lane == 0) {
        red_s[warp] = Us;
        red_c[warp] = Uc;
    }
    __syncthreads();
    if (warp == 0) {   // the warps' compensated partial sums, combined by a fixed butterfly
        float v = lane < W ? red_s[lane] - red_c[lane] : 0.0f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) *U_sh = v;
    }
    __syncthreads();
    return *U_sh;
}

// Gap current of local row rr (after gj_reduce).
template <int GJ>
__device__ __forceinline__ float row_current(const DenseSmem &sm, int rr, float u_i, int n, float U, float g) {
    float S = 0.0f;
#pragma unroll
    for (int k = 0; k < GJ; ++k) S += sm.part[rr * GJ + k];
    const float lin = fmaf((float)n, u_i, -U);
    return g * (1.0f / GJ_SCALE) * fmaf(0.8f, S, 0.2f * lin);
}

}  // namespace ion
