// ion_matrix.cu -- dense N x N weight-matrix connectivity (the programmed connectivity of
// Sec. 2.3 with every pair stored):
//   Ic_i = sum_j W[i][j] (0.8 e^{-dV^2/100} + 0.2) dV,  dV = V_dend,i - V_dend,j.
// The weights are stored padded to n_pad columns (zeros beyond n), so a padded column
// contributes exactly zero.  Every step streams the whole matrix from HBM (4 B per pair:
// 268 MB at 8192 cells), so the kernel is HBM-bound: a CTA of 8 warps owns 8 R rows,
// stages V_dend in tiles by bulk copy (as the uniform dense kernel does), and each lane
// reads, per float4 of columns, one 16-byte group of weights of each of its R rows
// (evict-first, 16 R bytes in flight per lane and load round).  Per-lane sums are folded
// with Kahan every BLK float4 groups and combined by a fixed butterfly (deterministic);
// the R rows' cell updates follow in the same launch.
#include <cuda_runtime.h>

#include "ion.h"
#include "ion_async.cuh"
#include "ion_dense_core.cuh"
#include "ion_kernels.cuh"

namespace ion {

template <int R>
__global__ void __launch_bounds__(256) matrix_step_kernel(const MatrixArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float part[8 * R];
    const StepCommon &c = a.c;
    const int n = c.n, n_pad = c.n_pad;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * 8 * R;
    constexpr int BLK = 8;   // float4 groups per lane between Kahan folds: a block is 32 * BLK groups (4 KB) per row
    const float *wrow[R];
#pragma unroll
    for (int r = 0; r < R; ++r) wrow[r] = a.W + (int64_t)min(row0 + warp * R + r, n - 1) * n_pad;   // rows past n: any row
    if (lane == 0)   // the weights are constant: their first two blocks are requested into L2 before the wait
#pragma unroll
        for (int r = 0; r < R; ++r) bulk_prefetch_l2(wrow[r], (uint32_t)min(2 * 32 * BLK * 16, n_pad * 4));
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    pdl_enter();
    __syncthreads();
    const int64_t t = step_index(c);
    const float *vcur = vd_cur(c);
    float *vnext = vd_next(c);
    const DenseSmem sm = dense_smem(smem_raw, n_pad);
    if (threadIdx.x == 0) {
        issue_tile(sm, vcur, n_pad, 0, bar);
        if (sm.n_tiles > 1) issue_tile(sm, vcur, n_pad, 1, bar);
    }
    const float m_shift = vcur[0];
    float ui[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = row0 + warp * R + r;
        ui[r] = row < n ? (vcur[row] - m_shift) * GJ_SCALE : 0.0f;
    }
    float ks[R], kc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) ks[r] = kc[r] = 0.0f;
    uint32_t uses[2] = {0u, 0u};
    const float2 c08 = make_float2(0.8f, 0.8f), c02 = make_float2(0.2f, 0.2f);
    for (int kt = 0; kt < sm.n_tiles; ++kt) {
        const int b = kt & 1;
        const int j0 = kt * TJ;
        const int len = min(TJ, n_pad - j0);
        const bool landed = mbar_wait_bounded(&bar[b], uses[b] & 1u);
        uses[b]++;
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) {   // wait (bounded) for the copies still in flight, then leave
                atomicOr(c.status, (uint32_t)ST_TIMEOUT);
                (void)mbar_wait_bounded(&bar[b], (uses[b] - 1u) & 1u);
                if (kt + 1 < sm.n_tiles) (void)mbar_wait_bounded(&bar[b ^ 1], uses[b ^ 1] & 1u);
            }
            return;
        }
        float *tb = sm.tile0 + b * sm.buf_len;
        for (int j = threadIdx.x; j < len; j += blockDim.x) {
            const bool real = j0 + j < n;
            tb[j] = real ? -(tb[j] - m_shift) * GJ_SCALE : -PAD_U;
        }
        __syncthreads();
        const float4 *t4 = reinterpret_cast<const float4 *>(tb);
        const int n4 = len >> 2;
        for (int m0 = lane; m0 < n4; m0 += 32 * BLK) {
            const int nb = m0 - lane + 2 * 32 * BLK;   // the block after next, requested into L2 now
            if (lane == 0 && nb < n4)
#pragma unroll
                for (int r = 0; r < R; ++r)
                    bulk_prefetch_l2(wrow[r] + j0 + 4 * nb, (uint32_t)min(32 * BLK, n4 - nb) * 16u);
            float2 acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = make_float2(0.0f, 0.0f);
            // the weights of the next group are requested before this group is computed
            float4 wn[R];
#pragma unroll
            for (int r = 0; r < R; ++r)
                wn[r] = m0 < n4 ? __ldcs(reinterpret_cast<const float4 *>(wrow[r] + j0) + m0) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
            for (int mm = 0; mm < BLK; ++mm) {
                const int mq = m0 + mm * 32;
                if (mq < n4) {
                    float4 w4[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) w4[r] = wn[r];
                    if (mm + 1 < BLK && mq + 32 < n4) {
#pragma unroll
                        for (int r = 0; r < R; ++r)
                            wn[r] = __ldcs(reinterpret_cast<const float4 *>(wrow[r] + j0) + mq + 32);
                    }
                    const float4 v = t4[mq];
                    const float2 va = make_float2(v.x, v.y), vb = make_float2(v.z, v.w);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float2 u2 = make_float2(ui[r], ui[r]);
                        const float2 da = __fadd2_rn(u2, va), db = __fadd2_rn(u2, vb);
                        const float2 qa = __fmul2_rn(da, da), qb = __fmul2_rn(db, db);
                        const float2 ea = make_float2(ex2_approx(-qa.x), ex2_approx(-qa.y));
                        const float2 eb = make_float2(ex2_approx(-qb.x), ex2_approx(-qb.y));
                        const float2 ta = __fmul2_rn(__ffma2_rn(ea, c08, c02), da);
                        const float2 tb2 = __fmul2_rn(__ffma2_rn(eb, c08, c02), db);
                        acc[r] = __ffma2_rn(ta, make_float2(w4[r].x, w4[r].y), acc[r]);
                        acc[r] = __ffma2_rn(tb2, make_float2(w4[r].z, w4[r].w), acc[r]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) kahan_add(ks[r], kc[r], acc[r].x + acc[r].y);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0 && kt + 2 < sm.n_tiles) issue_tile(sm, vcur, n_pad, kt + 2, bar);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float v = ks[r] - kc[r];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) part[warp * R + r] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x >= 8 * R) return;
    const int i = row0 + threadIdx.x;
    if (i >= n) return;
    const float ic = part[threadIdx.x] * (1.0f / GJ_SCALE);
    const Cell cell = load_cell(c.S, vcur, i);
    float iapp = pulse_current(c.pulses, i, t);
    if (c.iapp != nullptr) iapp += c.iapp[i];
    const CellNext o = cell_step(c.P, cell, ic, iapp);
    finish_cell(c, t, vnext, i, o);
}

size_t matrix_smem_bytes(int n_pad) { return (size_t)(n_pad > TJ ? 2 * TJ : n_pad) * sizeof(float); }

cudaError_t prepare_matrix_step(int n_pad) {
    const int smem = (int)matrix_smem_bytes(n_pad);
    cudaError_t e = cudaFuncSetAttribute(matrix_step_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(matrix_step_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(matrix_step_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

// rows per warp: the largest of 4, 2, 1 that still gives about six CTAs per SM (the
// weight stream needs many warps in flight; at 8192 cells R = 1 measured fastest), else 1
int matrix_default_R(int n, int sms) {
    for (int R : {4, 2})
        if ((n + 8 * R - 1) / (8 * R) >= 6 * sms) return R;
    return 1;
}

template <int R>
static cudaError_t matrix_launch_R(const MatrixArgs &a, cudaStream_t st) {
    const int grid = (a.c.n + 8 * R - 1) / (8 * R);
    return launch_k(matrix_step_kernel<R>, dim3(grid), dim3(256), matrix_smem_bytes(a.c.n_pad), st, a.c.pdl != 0, a);
}
cudaError_t launch_matrix_step(const MatrixArgs &a, int R, cudaStream_t st) {
    switch (R) {
        case 1: return matrix_launch_R<1>(a, st);
        case 2: return matrix_launch_R<2>(a, st);
        case 4: return matrix_launch_R<4>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ion
