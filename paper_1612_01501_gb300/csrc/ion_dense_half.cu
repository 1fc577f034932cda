// ion_dense_half.cu -- persistent dense step that evaluates each unordered pair once.
//
// The gap-junction term is odd, T(-dV) = -T(dV), and a dense network has one weight for
// every pair, so I_ij = -I_ji: a pair evaluated once serves both cells.  With G CTAs, CTA c
// owns rows block c (b rows) and takes as columns its own block and the next D blocks
// (c+1 .. c+D mod G, D = (G-1)/2, plus block c + G/2 for c < G/2 when G is even), so every
// unordered pair of blocks is evaluated by exactly one CTA.  In one pass over its column
// tile each lane accumulates the row sums of its R rows (as in the full-work kernels) and,
// for every column, the sum over those rows; the column sums of the R-row groups are then
// reduced in a fixed order and written to an L2-resident buffer.  After a grid barrier
// each CTA gathers, for its own rows, the negated column sums the other CTAs computed for
// them (in a fixed order), adds its row sums and the closed-form linear part, runs the
// cell update and writes V_dend(t+1); a second barrier ends the step.  Per pair: one FADD2,
// one FMUL2, two ex2, two FFMA2 for two pairs -- half the SFU work of the full pass.
//
// Cell state stays in registers across steps, as in the full-work persistent kernel.
#include <cuda_runtime.h>

#include "ion_async.cuh"
#include "ion_kernels.cuh"

namespace ion {

constexpr float HALF_PAD_U = 1.0e6f;   // 2^{-PAD^2} is exactly 0
constexpr int HALF_LOADS = 8;          // independent loads in flight per thread when gathering or reducing
constexpr int HALF_SMEM_BUDGET = 220 * 1024;   // dynamic shared memory per CTA (one CTA per SM)

__device__ __forceinline__ int half_partners(int c, int G) {   // D_c: blocks after c taken as columns
    const int D = (G - 1) / 2;
    return D + ((G % 2 == 0 && c < G / 2) ? 1 : 0);
}
__device__ __forceinline__ bool half_has(int src, int d, int G) {   // does CTA src take block src + d?
    return d >= 1 && d <= half_partners(src, G);
}

template <int R, int GJ>
__global__ void __launch_bounds__(896) dense_half_kernel(const HalfArgs a) {
    extern __shared__ __align__(16) float hsm[];
    __shared__ float red_s[32], red_c[32];
    __shared__ float U_sh;
    __shared__ int ok_sh;

    const StepCommon &c = a.c;
    const int n = c.n, G = gridDim.x, b = a.rows;
    const int W = blockDim.x >> 5, GR = W / GJ;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rg = warp % GR, cs = warp / GR;
    const int cta = blockIdx.x;
    const int P = G * b;                                    // padded row space
    const int Dc = half_partners(cta, G);
    const int L = (Dc + 1) * b;                            // own block + D_c partner blocks
    const int Lp = (L + 127) / 128 * 128;                   // whole float4 rounds of 32 lanes
    const int CH = a.chunk;                                 // tile columns per column-partial round
    float *tile = hsm;                                      // [a.colsum_stride]  -u_j of the column tile
    float *colpart = tile + a.colsum_stride;                // [GR][CH]
    float *part = colpart + GR * CH;                        // [b] row sums of own rows
    float *colsum_me = a.colsum + (int64_t)cta * a.colsum_stride;

    const int row0 = cta * b;
    const int my_row = row0 + (int)threadIdx.x;
    const bool row_thread = (int)threadIdx.x < b && my_row < n;
    const int64_t t0 = *c.t_dev;
    Cell cell{};
    float o_ms = 0.0f, o_ma = 0.0f, o_icah = 0.0f, o_ic = 0.0f;
    int32_t p0 = 0, p1 = 0;
    if (row_thread) {
        cell = load_cell(c.S, vd_slot(c.S, t0), my_row);
        if (c.pulses.off != nullptr) {
            p0 = c.pulses.off[my_row];
            p1 = c.pulses.off[my_row + 1];
        }
    }
    if (a.debug_delay_ns > 0 && cta == G - 1 && threadIdx.x == 0) {
        const uint64_t d0 = globaltimer_ns();
        while (globaltimer_ns() - d0 < (uint64_t)a.debug_delay_ns) __nanosleep(1000);
    }

    bool ok = true;
    uint32_t bar_target = a.bar_base;
    for (int k = 0; k < a.n_steps && ok; ++k) {
        const int64_t t = t0 + k;
        const float *vcur = vd_slot(c.S, t);
        const float m = __ldcg(vcur);      // the shift, loaded by every thread with its tile loads
        // stage the column tile: own block, then the partner blocks (wrapping), as -u;
        // HALF_LOADS loads per thread are issued before any is used
        float Us = 0.0f, Uc = 0.0f;   // this thread's share of the own block's sum of u
        for (int q0 = 0; q0 < Lp; q0 += HALF_LOADS * (int)blockDim.x) {
            float vv[HALF_LOADS];
#pragma unroll
            for (int j = 0; j < HALF_LOADS; ++j) {
                const int q = q0 + j * (int)blockDim.x + (int)threadIdx.x;
                const int row = (row0 + q) % P;
                vv[j] = (q < L && row < n) ? __ldcg(vcur + row) : 0.0f;
            }
#pragma unroll
            for (int j = 0; j < HALF_LOADS; ++j) {
                const int q = q0 + j * (int)blockDim.x + (int)threadIdx.x;
                if (q < Lp) {
                    float v = -HALF_PAD_U;
                    if (q < L && (row0 + q) % P < n) {
                        const float u = (vv[j] - m) * GJ_SCALE;
                        v = -u;
                        if (q < b) kahan_add(Us, Uc, u);
                    }
                    tile[q] = v;
                }
            }
        }
        __syncthreads();
        float ui[R];
#pragma unroll
        for (int r = 0; r < R; ++r) ui[r] = -tile[rg * R + r];   // own rows (phantom rows: -PAD)
        float ks[R], kc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) ks[r] = kc[r] = 0.0f;
        const float4 *t4 = reinterpret_cast<const float4 *>(tile);
        for (int ch = 0; ch * CH < Lp; ++ch) {
            const int nq = min(CH, Lp - ch * CH);                   // columns in this chunk
            const int G4 = nq / 4;                                  // float4 columns
            float2 acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = make_float2(0.0f, 0.0f);
            for (int m4 = cs * 32 + lane; m4 < G4; m4 += 32 * GJ) {
                const float4 v = t4[ch * (CH / 4) + m4];
                const float2 va = make_float2(v.x, v.y), vb = make_float2(v.z, v.w);
                float2 ca = make_float2(0.0f, 0.0f), cb = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 u2 = make_float2(ui[r], ui[r]);
                    const float2 da = __fadd2_rn(u2, va);
                    const float2 db = __fadd2_rn(u2, vb);
                    const float2 qa = __fmul2_rn(da, da);
                    const float2 qb = __fmul2_rn(db, db);
                    const float2 ea = make_float2(ex2_approx(-qa.x), ex2_approx(-qa.y));
                    const float2 eb = make_float2(ex2_approx(-qb.x), ex2_approx(-qb.y));
                    acc[r] = __ffma2_rn(ea, da, acc[r]);
                    acc[r] = __ffma2_rn(eb, db, acc[r]);
                    ca = __ffma2_rn(ea, da, ca);
                    cb = __ffma2_rn(eb, db, cb);
                }
                reinterpret_cast<float4 *>(colpart + rg * CH)[m4] = make_float4(ca.x, ca.y, cb.x, cb.y);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) kahan_add(ks[r], kc[r], acc[r].x + acc[r].y);
            __syncthreads();
            // column sums of this chunk: the R-row groups summed in ascending order (loads
            // issued HALF_LOADS at a time)
            for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                float s = 0.0f;
                int g = 0;
                for (; g + HALF_LOADS <= GR; g += HALF_LOADS) {
                    float v[HALF_LOADS];
#pragma unroll
                    for (int j = 0; j < HALF_LOADS; ++j) v[j] = colpart[(g + j) * CH + q];
#pragma unroll
                    for (int j = 0; j < HALF_LOADS; ++j) s += v[j];
                }
                for (; g < GR; ++g) s += colpart[g * CH + q];
                colsum_me[ch * CH + q] = s;
            }
            __syncthreads();
        }
        // own row sums: butterfly over lanes, then the column splits
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float v = ks[r] - kc[r];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0 && cs == 0) part[rg * R + r] = v;
            if (GJ > 1) {
                __syncthreads();
                for (int s2 = 1; s2 < GJ; ++s2) {
                    if (lane == 0 && cs == s2) part[rg * R + r] += v;
                    __syncthreads();
                }
            }
        }
        // this CTA's sum of u over its own rows -> a.usum[cta]
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
        if (threadIdx.x == 0) {
            float s = 0.0f, cc = 0.0f;
            for (int w = 0; w < W; ++w) kahan_add(s, cc, red_s[w] - red_c[w]);
            a.usum[cta] = s - cc;
        }
        // barrier A: every column sum and partial sum of u of this step is written
        bar_target += G;
        ok = grid_barrier(a.bar_count, a.abort_flag, bar_target, a.timeout_ns, c.status, &ok_sh);
        if (!ok) break;
        // sum of u over all cells: warp 0, lane-strided Kahan sums then a butterfly
        if (warp == 0) {
            float s = 0.0f, cc = 0.0f;
            for (int q0 = 0; q0 < G; q0 += 32 * HALF_LOADS) {
                float vv[HALF_LOADS];
#pragma unroll
                for (int j = 0; j < HALF_LOADS; ++j) {
                    const int q = q0 + 32 * j + lane;
                    vv[j] = q < G ? __ldcg(a.usum + q) : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < HALF_LOADS; ++j) kahan_add(s, cc, vv[j]);
            }
            float v = s - cc;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) U_sh = v;
        }
        // the negated column sums other CTAs computed for this block: CTA cta - d took it at
        // distance d; all threads load them (HALF_LOADS in flight each) into shared memory,
        // then each row thread adds them in ascending d (0 where the source did not take it)
        const int r = threadIdx.x;
        float s = row_thread ? part[r] : 0.0f, cc = 0.0f;
        const int slab = (GR * CH) / b;                 // distances per round (>= 128 / R)
        for (int d0 = 1; d0 <= G / 2; d0 += slab) {
            const int nd = min(slab, G / 2 - d0 + 1), tot = nd * b;
            for (int i0 = 0; i0 < tot; i0 += HALF_LOADS * (int)blockDim.x) {
                float vv[HALF_LOADS];
#pragma unroll
                for (int j = 0; j < HALF_LOADS; ++j) {
                    const int idx = i0 + j * (int)blockDim.x + (int)threadIdx.x;
                    const int d = d0 + idx / b, src = (cta - d + G) % G;
                    vv[j] = (idx < tot && half_has(src, d, G))
                                ? __ldcg(a.colsum + (int64_t)src * a.colsum_stride + d * b + idx % b)
                                : 0.0f;
                }
#pragma unroll
                for (int j = 0; j < HALF_LOADS; ++j) {
                    const int idx = i0 + j * (int)blockDim.x + (int)threadIdx.x;
                    if (idx < tot) colpart[idx] = vv[j];
                }
            }
            __syncthreads();
            if (row_thread) {
                int dd = 0;
                for (; dd + HALF_LOADS <= nd; dd += HALF_LOADS) {
                    float v[HALF_LOADS];
#pragma unroll
                    for (int j = 0; j < HALF_LOADS; ++j) v[j] = colpart[(dd + j) * b + r];
#pragma unroll
                    for (int j = 0; j < HALF_LOADS; ++j) kahan_add(s, cc, -v[j]);
                }
                for (; dd < nd; ++dd) kahan_add(s, cc, -colpart[dd * b + r]);
            }
            __syncthreads();
        }
        if (row_thread) {
            const float S = s - cc;
            const float u_i = (cell.vd - m) * GJ_SCALE;
            const float lin = fmaf((float)n, u_i, -U_sh);
            const float ic = a.g * (1.0f / GJ_SCALE) * fmaf(0.8f, S, 0.2f * lin);
            float iapp = 0.0f;
            for (int32_t p = p0; p < p1; ++p)
                if (t >= c.pulses.begin[p] && t < c.pulses.end[p]) iapp += c.pulses.amp[p];
            const CellNext o = cell_step(c.P, cell, ic, iapp);
            cell.vd = o.vd; cell.vs = o.vs; cell.va = o.va; cell.ca = o.ca;
            cell.r = o.r; cell.s = o.s; cell.q = o.q; cell.k = o.k; cell.l = o.l;
            cell.hs = o.hs; cell.ns = o.ns; cell.xs = o.xs; cell.ha = o.ha; cell.xa = o.xa;
            o_ms = o.ms; o_ma = o.ma; o_icah = o.icah; o_ic = o.ic;
            if (!cell_finite(o)) atomicOr(c.status, (uint32_t)ST_NONFINITE);
            if (c.trace != nullptr && ((t + 1) % c.trace_stride) == 0) {
                const int64_t sample = (t + 1) / c.trace_stride - 1;
                c.trace[(sample % c.trace_cap) * (int64_t)n + my_row] = o.va;
            }
            vd_slot(c.S, t + 1)[my_row] = cell.vd;
        }
        // barrier B: V_dend(t+1) is complete (and every read of this step's sums is done)
        bar_target += G;
        ok = grid_barrier(a.bar_count, a.abort_flag, bar_target, a.timeout_ns, c.status, &ok_sh);
    }
    if (row_thread && a.n_steps > 0) {
        const CellNext o{cell.vd, cell.vs, cell.va, cell.ca, cell.r, cell.s, cell.q, cell.k, cell.l, o_ms,
                         cell.hs, cell.ns, cell.xs, o_ma, cell.ha, cell.xa, o_icah, o_ic};
        store_cell(c.S, vd_slot(c.S, t0 + a.n_steps), my_row, o);
    }
}

// longest column tile (own block + the most partner blocks), in whole rounds of 128 columns
int half_colsum_stride(int G, int b) {
    const int D = (G - 1) / 2 + ((G % 2 == 0) ? 1 : 0);
    return ((D + 1) * b + 127) / 128 * 128;
}
// columns per column-partial round: the fewest rounds whose partials fit the budget, split
// evenly in multiples of 128
int half_chunk(int G, int b, int GR) {
    const int stride = half_colsum_stride(G, b);
    const int room = HALF_SMEM_BUDGET / (int)sizeof(float) - stride - b;
    const int max_ch = room / GR / 128 * 128;
    if (max_ch < 128) return 0;
    const int rounds = (stride + max_ch - 1) / max_ch;
    const int ch = ((stride + rounds - 1) / rounds + 127) / 128 * 128;
    return ch < max_ch ? ch : max_ch;
}
size_t half_smem_bytes(int G, int b, int GR, int CH) {
    return (size_t)(half_colsum_stride(G, b) + GR * CH + b) * sizeof(float);
}

template <int R, int GJ>
static cudaError_t half_RG(const HalfArgs &a0, int W, int G, bool launch, int *ok_out, cudaStream_t st) {
    const int GR = W / GJ;
    HalfArgs a = a0;
    a.chunk = half_chunk(G, a.rows, GR);
    if (a.chunk < 128) {
        *ok_out = 0;
        return launch ? cudaErrorInvalidValue : cudaSuccess;
    }
    const size_t smem = half_smem_bytes(G, a.rows, GR, a.chunk);
    if (!launch) {
        cudaError_t e = cudaFuncSetAttribute(dense_half_kernel<R, GJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense_half_kernel<R, GJ>, W * 32, smem);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        *ok_out = (G <= per_sm * sms) ? 1 : 0;
        return cudaSuccess;
    }
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel((const void *)dense_half_kernel<R, GJ>, dim3(G), dim3(W * 32), args, smem, st);
}

// rows per CTA = a.rows = (W / GJ) * R; grid G CTAs (every CTA resident).  launch false:
// prepare and report in *ok_out whether the grid fits at once.
cudaError_t launch_dense_half(const HalfArgs &a, int R, int W, int GJ, int G, bool launch, int *ok_out,
                              cudaStream_t st) {
    int dummy = 0;
    if (!ok_out) ok_out = &dummy;
    if (W < 1 || W > 28 || (GJ != 1 && GJ != 2) || W % GJ != 0 || (W / GJ) * R != a.rows || G < 2)
        return cudaErrorInvalidValue;
    switch (R) {
        case 1: return GJ == 1 ? half_RG<1, 1>(a, W, G, launch, ok_out, st) : half_RG<1, 2>(a, W, G, launch, ok_out, st);
        case 2: return GJ == 1 ? half_RG<2, 1>(a, W, G, launch, ok_out, st) : half_RG<2, 2>(a, W, G, launch, ok_out, st);
        case 4: return GJ == 1 ? half_RG<4, 1>(a, W, G, launch, ok_out, st) : half_RG<4, 2>(a, W, G, launch, ok_out, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ion
