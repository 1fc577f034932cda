// ion_csr.cu -- sparse (CSR) gap-junction step and the stand-alone cell update.
//
// Algorithm 1 over a programmed weight matrix (Sec. 2.3): for every stored connection
// e = (i, j) of row i,
//   Ic_i += w_e (0.8 e^{-dV^2/100} + 0.2) dV,  dV = V_dend,i - V_dend,j.
// One CTA owns `rows_per_cta` consecutive rows (= its thread count).  Phase 1: groups of
// SW lanes (SW = 1..32, picked from the mean degree) walk one row's edges with a stride
// of SW, so the index and weight loads of a group are contiguous; four edges per lane
// are in flight per iteration to hide the latency of the V_dend gathers; the SW lane
// sums are combined with shuffles in a fixed order.  Phase 2: one thread per row runs
// the explicit-Euler cell update with that row's current (fused variant), so the cell
// work runs on full warps whatever SW is.
#include <cuda_runtime.h>

#include "ion_kernels.cuh"

namespace ion {

__device__ __forceinline__ float gj_edge(float vi, float vj, float w) {
    const float du = (vi - vj) * GJ_SCALE;
    return w * fmaf(0.8f, ex2_approx(-du * du), 0.2f) * du;
}

template <int SW>
__global__ void __launch_bounds__(1024) csr_step_kernel(const CsrArgs a) {
    extern __shared__ float ic_s[];
    const StepCommon &c = a.c;
    const int n = c.n;
    const int rows_cta = blockDim.x;
    const int row0 = blockIdx.x * rows_cta;
    const int64_t t = step_index(c);
    const float *vcur = a.vd_in != nullptr ? a.vd_in : vd_cur(c, t);
    float *vnext = a.fuse ? vd_next(c, t) : nullptr;
    const int sub = threadIdx.x / SW, li = threadIdx.x % SW, nsub = blockDim.x / SW;
    const float *__restrict__ w = a.w;
    const int32_t *__restrict__ col = a.col;

    for (int rr = sub; rr < rows_cta; rr += nsub) {   // SW iterations for every lane
        const int i = row0 + rr;
        float acc = 0.0f;
        if (i < n) {
            const float vi = vcur[i];
            const int e1 = a.row_ptr[i + 1];
            int e = a.row_ptr[i] + li;
            if (w != nullptr) {
                for (; e + 3 * SW < e1; e += 4 * SW) {
                    const int j0 = __ldg(col + e), j1 = __ldg(col + e + SW), j2 = __ldg(col + e + 2 * SW),
                              j3 = __ldg(col + e + 3 * SW);
                    const float w0 = __ldg(w + e), w1 = __ldg(w + e + SW), w2 = __ldg(w + e + 2 * SW),
                                w3 = __ldg(w + e + 3 * SW);
                    const float v0 = __ldg(vcur + j0), v1 = __ldg(vcur + j1), v2 = __ldg(vcur + j2),
                                v3 = __ldg(vcur + j3);
                    acc += gj_edge(vi, v0, w0) + gj_edge(vi, v1, w1) + (gj_edge(vi, v2, w2) + gj_edge(vi, v3, w3));
                }
                for (; e < e1; e += SW) acc += gj_edge(vi, __ldg(vcur + __ldg(col + e)), __ldg(w + e));
            } else {
                for (; e + 3 * SW < e1; e += 4 * SW) {
                    const int j0 = __ldg(col + e), j1 = __ldg(col + e + SW), j2 = __ldg(col + e + 2 * SW),
                              j3 = __ldg(col + e + 3 * SW);
                    const float v0 = __ldg(vcur + j0), v1 = __ldg(vcur + j1), v2 = __ldg(vcur + j2),
                                v3 = __ldg(vcur + j3);
                    acc += gj_edge(vi, v0, 1.0f) + gj_edge(vi, v1, 1.0f) +
                           (gj_edge(vi, v2, 1.0f) + gj_edge(vi, v3, 1.0f));
                }
                for (; e < e1; e += SW) acc += gj_edge(vi, __ldg(vcur + __ldg(col + e)), 1.0f);
                acc *= a.g;
            }
        }
#pragma unroll
        for (int off = SW / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (li == 0 && i < n) ic_s[rr] = acc * (1.0f / GJ_SCALE);
    }
    __syncthreads();
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

template <int SW>
static cudaError_t launch_csr_SW(const CsrArgs &a, int rows, cudaStream_t st) {
    const int grid = (a.c.n + rows - 1) / rows;
    csr_step_kernel<SW><<<grid, rows, rows * sizeof(float), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_csr_step(const CsrArgs &a, int SW, int rows, cudaStream_t st) {
    if (rows < 32 || rows > 1024 || rows % 32 != 0) return cudaErrorInvalidValue;
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

// ---- stand-alone cell update (no gap junctions, or Ic computed by another launch) ----
__global__ void __launch_bounds__(256) cell_step_kernel(const CellArgs a) {
    const StepCommon &c = a.c;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n) return;
    const int64_t t = step_index(c);
    const float *vcur = vd_cur(c, t);
    float *vnext = vd_next(c, t);
    const Cell cell = load_cell(c.S, vcur, i);
    const float ic = a.ic != nullptr ? a.ic[i] : 0.0f;
    float iapp = pulse_current(c.pulses, i, t);
    if (c.iapp != nullptr) iapp += c.iapp[i];
    const CellNext o = cell_step(c.P, cell, ic, iapp);
    finish_cell(c, t, vnext, i, o);
}

cudaError_t launch_cell_step(const CellArgs &a, cudaStream_t st) {
    const int64_t grid = ((int64_t)a.c.n + 255) / 256;
    cell_step_kernel<<<(unsigned)grid, 256, 0, st>>>(a);
    return cudaGetLastError();
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
