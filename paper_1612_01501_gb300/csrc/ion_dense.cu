// ion_dense.cu -- dense all-to-all gap-junction step (Algorithm 1 with C = 100 %).
//
// For a uniform pair weight g the gap current of cell i is
//   Ic_i = g sum_j (0.8 e^{-dV_ij^2/100} + 0.2) dV_ij,  dV_ij = V_i - V_j   (j = 0..N-1).
// With u = s V, s = sqrt(log2(e)/100), the exponential is 2^{-(u_i-u_j)^2} (one SFU ex2),
// and the linear part sums in closed form: sum_j dV_ij = N V_i - sum_j V_j.  So
//   Ic_i = (g/s) [0.8 sum_j 2^{-du^2} du + 0.2 (N u_i - sum_j u_j)],  du = u_i - u_j,
// and each pair costs one FADD, one FMUL, one ex2 and one FFMA.
//
// Layout of one launch (N-body style): V_dend(t) is staged into shared memory in tiles
// of TJ floats by 1-D bulk async copies (cp.async.bulk, completion on an mbarrier),
// double-buffered when N > TJ.  A CTA owns W*R consecutive rows; each warp owns R of
// them and each lane walks the tile 4 columns at a time (one 16-byte shared load feeds
// 4 x R pairs).  Lane sums are folded into Kahan-compensated accumulators every 64
// columns; after the last tile the 32 lane partials of each row go to shared memory
// and the thread that updates the row sums them (again compensated) in a fixed order,
// so results are deterministic.  The fused variant then runs the explicit-Euler cell
// update of the CTA's rows (one thread per row) and writes V_dend(t+1) to the other
// buffer, so one launch is one whole step.
#include <cuda_runtime.h>

#include "ion_kernels.cuh"

namespace ion {

// ---- mbarrier + bulk-copy helpers (sm_90+ PTX) ------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait on an mbarrier phase: gives up after ~0.5 s (then flags ST_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase) {
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, phase)) return true;
        if ((it & 255u) == 255u && globaltimer_ns() - t0 > 500000000ull) break;
    }
    return mbar_try_wait(bar, phase);
}
// 1-D bulk copy global -> shared, completion counted in bytes on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// ---- the kernel -------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(512) dense_step_kernel(const DenseArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float red_s[32], red_c[32];
    __shared__ float U_sh;

    const StepCommon &c = a.c;
    const int n = c.n;
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rows_cta = W * R;
    const int n_tiles = (c.n_pad + TJ - 1) / TJ;
    const int buf_len = n_tiles > 1 ? TJ : c.n_pad;
    float *const tile0 = reinterpret_cast<float *>(smem_raw);    // buffer b at tile0 + b * buf_len
    float *part_s = tile0 + (n_tiles > 1 ? 2 * TJ : c.n_pad);    // [rows_cta][33]
    float *part_c = part_s + rows_cta * 33;

    const int64_t t = step_index(c);
    const float *vcur = a.vd_in != nullptr ? a.vd_in : vd_cur(c, t);
    float *vnext = a.fuse ? vd_next(c, t) : nullptr;
    const int row_base = blockIdx.x * rows_cta;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 2 && k < n_tiles; ++k) {
            const int len = min(TJ, c.n_pad - k * TJ);
            mbar_expect_tx(&bar[k], (uint32_t)len * 4u);
            bulk_g2s(tile0 + k * buf_len, vcur + (int64_t)k * TJ, (uint32_t)len * 4u, &bar[k]);
        }
    }

    // rows of this lane (scaled voltages), read directly from global memory
    float ui[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = row_base + warp * R + r;
        ui[r] = (i < n) ? vcur[i] * GJ_SCALE : 0.0f;
    }
    float ks[R], kc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) ks[r] = kc[r] = 0.0f;
    float Us = 0.0f, Uc = 0.0f;   // this thread's share of sum_j u_j (compensated)

    bool ok = true;
    for (int kt = 0; kt < n_tiles; ++kt) {
        const int b = kt & 1;
        const int j0 = kt * TJ;
        const int len = min(TJ, c.n_pad - j0);
        const bool landed = mbar_wait_bounded(&bar[b], (uint32_t)((kt >> 1) & 1));
        if (__syncthreads_or(!landed)) {   // block-uniform decision
            ok = false;
            break;
        }
        // scale the tile in place and accumulate this thread's part of sum_j u_j
        float *tb = tile0 + b * buf_len;
        for (int j = threadIdx.x; j < len; j += blockDim.x) {
            const float u = tb[j] * GJ_SCALE;
            tb[j] = u;
            if (j0 + j < n) kahan_add(Us, Uc, u);
        }
        __syncthreads();
        const float4 *t4 = reinterpret_cast<const float4 *>(tb);
        const int n4 = len >> 2;             // float4 columns; len is a multiple of 256
        for (int m0 = lane; m0 < n4; m0 += 32 * 16) {
            float acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = 0.0f;
#pragma unroll 4
            for (int mm = 0; mm < 16; ++mm) {
                const int m = m0 + mm * 32;
                if (m < n4) {
                    const float4 v = t4[m];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float d0 = ui[r] - v.x, d1 = ui[r] - v.y, d2 = ui[r] - v.z, d3 = ui[r] - v.w;
                        acc[r] = fmaf(ex2_approx(-d0 * d0), d0, acc[r]);
                        acc[r] = fmaf(ex2_approx(-d1 * d1), d1, acc[r]);
                        acc[r] = fmaf(ex2_approx(-d2 * d2), d2, acc[r]);
                        acc[r] = fmaf(ex2_approx(-d3 * d3), d3, acc[r]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (a.kahan) kahan_add(ks[r], kc[r], acc[r]);
                else ks[r] += acc[r];
            }
        }
        __syncthreads();   // every thread is done with this buffer
        if (threadIdx.x == 0 && kt + 2 < n_tiles) {
            // order this CTA's generic-proxy accesses of the buffer before the async refill
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const int len2 = min(TJ, c.n_pad - (kt + 2) * TJ);
            mbar_expect_tx(&bar[b], (uint32_t)len2 * 4u);
            bulk_g2s(tb, vcur + (int64_t)(kt + 2) * TJ, (uint32_t)len2 * 4u, &bar[b]);
        }
    }
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicOr(c.status, (uint32_t)ST_TIMEOUT);
            // let any copy still in flight land before the CTA's shared memory is released
            for (int k = 0; k < 2 && k < n_tiles; ++k) (void)mbar_wait_bounded(&bar[k], 0);
        }
        return;
    }

    // lane partials of each row -> shared memory
#pragma unroll
    for (int r = 0; r < R; ++r) {
        part_s[(warp * R + r) * 33 + lane] = ks[r];
        part_c[(warp * R + r) * 33 + lane] = kc[r];
    }
    // sum_j u_j: warp partials (plain shuffle sum of the compensated thread sums is
    // carried as separate sum / compensation channels), then warp 0 finishes
    float s1 = Us, c1 = Uc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        c1 += __shfl_xor_sync(0xffffffffu, c1, off);
    }
    if (lane == 0) {
        red_s[warp] = s1;
        red_c[warp] = c1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f, cc = 0.0f;
        for (int w = 0; w < W; ++w) kahan_add(s, cc, red_s[w] - red_c[w]);
        U_sh = s - cc;
    }
    __syncthreads();
    const float U = U_sh;
    const float g_over_s = a.g * (1.0f / GJ_SCALE);

    for (int rr = threadIdx.x; rr < rows_cta; rr += blockDim.x) {
        const int i = row_base + rr;
        if (i >= n) break;
        float s = 0.0f, cc = 0.0f;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) {
            kahan_add(s, cc, part_s[rr * 33 + l]);
            kahan_add(s, cc, -part_c[rr * 33 + l]);
        }
        const float S = s - cc;
        const float u_i = vcur[i] * GJ_SCALE;
        const float lin = fmaf((float)n, u_i, -U);
        const float ic = g_over_s * fmaf(0.8f, S, 0.2f * lin);
        if (!a.fuse) {
            a.ic_out[i] = ic;
            continue;
        }
        const Cell cell = load_cell(c.S, vcur, i);
        float iapp = pulse_current(c.pulses, i, t);
        if (c.iapp != nullptr) iapp += c.iapp[i];
        const CellNext o = cell_step(c.P, cell, ic, iapp);
        finish_cell(c, t, vnext, i, o);
    }
}

size_t dense_smem_bytes(int n_pad, int R, int W) {
    const int n_tiles = (n_pad + TJ - 1) / TJ;
    const size_t tiles = (n_tiles > 1 ? 2 * TJ : n_pad) * sizeof(float);
    return tiles + 2 * (size_t)W * R * 33 * sizeof(float);
}

template <int R>
static cudaError_t launch_dense_R(const DenseArgs &a, int W, cudaStream_t st) {
    const int rows_cta = W * R;
    const int grid = (a.c.n + rows_cta - 1) / rows_cta;
    const size_t smem = dense_smem_bytes(a.c.n_pad, R, W);
    dense_step_kernel<R><<<grid, W * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int R>
static cudaError_t prepare_dense_R(int W, int n_pad) {
    const size_t smem = dense_smem_bytes(n_pad, R, W);
    return cudaFuncSetAttribute(dense_step_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Raise the kernel's dynamic shared-memory limit (done once, outside stream capture).
cudaError_t prepare_dense_step(int R, int W, int n_pad) {
    switch (R) {
        case 1: return prepare_dense_R<1>(W, n_pad);
        case 2: return prepare_dense_R<2>(W, n_pad);
        case 4: return prepare_dense_R<4>(W, n_pad);
        case 6: return prepare_dense_R<6>(W, n_pad);
        case 8: return prepare_dense_R<8>(W, n_pad);
        default: return cudaErrorInvalidValue;
    }
}
int dense_max_rows_per_warp() { return 8; }

cudaError_t launch_dense_step(const DenseArgs &a, int R, int W, cudaStream_t st) {
    switch (R) {
        case 1: return launch_dense_R<1>(a, W, st);
        case 2: return launch_dense_R<2>(a, W, st);
        case 4: return launch_dense_R<4>(a, W, st);
        case 6: return launch_dense_R<6>(a, W, st);
        case 8: return launch_dense_R<8>(a, W, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ion
