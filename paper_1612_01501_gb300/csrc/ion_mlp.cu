// ion_mlp.cu -- learned surrogate of the channel rate functions (not in the paper).
//
// A small MLP, (V, [Ca]) -> 64 tanh -> 64 tanh -> 24 outputs, stands in for the gates'
// rate functions: output 2g is logit(x_inf) of gate g (clipped to +-LOGIT_MAX), output 2g+1
// is ln(tau) (the instantaneous gates m_s, m_a have no tau; that output is masked out of
// the loss).  The logit keeps small steady states (m_inf^3 of the Na channels near rest)
// accurate in relative terms; a first fit of x_inf itself made resting cells fire.  Inputs
// and outputs are normalised (shift / scale kept with the weights).
//
// Training (ion_surrogate_train): samples V uniform in [v_lo, v_hi] and [Ca] log-uniform
// are drawn on the device (splitmix64 in counter form, Steele-Lea-Flood 2014), labelled
// by the exact FP32 rate functions of ion_model.cuh, and fitted by minibatch Adam.  Each
// minibatch is one launch of mlp_grad_kernel (128 samples per CTA; forward and backward
// in FP32 with activations in shared memory; each CTA writes its partial gradient) and
// one launch of mlp_adam_kernel (sums the partials in a fixed order, then the Adam step
// on FP32 master weights), so training is deterministic.
//
// Inference runs on the tensor cores, BF16 weights and activations with FP32 accumulation:
// by default on tcgen05 with TMEM accumulators (ion_mlp_tc.cu: ion_surrogate_eval and the
// cell update); with ION_FLAG_SURROGATE_WARP_MMA the cell update below uses mma.sync
// m16n8k16 instead (kept for comparison).  Layer 1 (two
// inputs) is FP32 FMAs; the 64x64 and 64x24 layers are MMAs whose accumulator fragments
// become the next layer's A fragments in registers; tanh runs on packed bf16 pairs.
// The cell kernel evaluates one row per (cell, compartment) -- 96 rows per warp for 32
// cells -- then each lane runs the explicit-Euler update of one cell with those rates.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "ion.h"
#include "ion_kernels.cuh"
#include "ion_sim.h"

namespace ion {

constexpr int MI = ION_MLP_IN, MH = ION_MLP_HID, MO = ION_MLP_OUT;
constexpr int P_W1 = 0, P_B1 = P_W1 + MH * MI, P_W2 = P_B1 + MH, P_B2 = P_W2 + MH * MH, P_W3 = P_B2 + MH,
              P_B3 = P_W3 + MO * MH, P_TOTAL = P_B3 + MO;   // 5912 parameters, the order of ion_surrogate_weights
constexpr int MB = 128;                                      // samples per CTA in training
constexpr int HS = MH + 1;                                   // padded row stride of activation tiles
constexpr float V_CENTER = -25.0f, V_HALF = 75.0f;
constexpr float LOGIT_MAX = 15.0f;

// ---- counter-based generator (splitmix64) --------------------------------------------
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double sm64_uniform(uint64_t seed, uint64_t k) {
    return (double)(sm64_mix(seed + (k + 1) * 0x9E3779B97F4A7C15ull) >> 11) * (1.0 / 9007199254740992.0);
}

// ---- data: samples, exact targets, normalisation ---------------------------------------
__global__ void mlp_samples_kernel(int64_t n, uint64_t seed, float v_lo, float v_hi, float lc_lo, float lc_hi, float *V,
                                   float *ca) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint64_t sa = sm64_mix(seed + 0x9E3779B97F4A7C15ull), sb = sm64_mix(seed + 2 * 0x9E3779B97F4A7C15ull);
    V[k] = (float)(v_lo + (v_hi - v_lo) * sm64_uniform(sa, (uint64_t)k));
    ca[k] = (float)exp(lc_lo + (lc_hi - lc_lo) * sm64_uniform(sb, (uint64_t)k));
}

// raw targets of one (V, ca): logit(x_inf) and ln(tau) of every gate (ln tau = 0 for the
// instantaneous ones)
__device__ __forceinline__ void exact_targets(float V, float ca, float *out) {
    const Rate g[NG] = {rate_r(V), rate_s(ca), rate_q(V), rate_k(V), rate_l(V), {minf_na(V), 0.0f},
                        rate_hs(V), rate_ns(V), rate_x(V), {minf_na(V), 0.0f}, rate_ha(V), rate_x(V)};
    for (int k = 0; k < NG; ++k) {
        const float x = fminf(fmaxf(g[k].xinf, 1e-30f), 1.0f);
        const float lg = logf(x) - log1pf(-fminf(x, 1.0f - 1e-7f));
        out[2 * k] = fminf(fmaxf(lg, -LOGIT_MAX), LOGIT_MAX);
        out[2 * k + 1] = g[k].inv_tau > 0.0f ? -logf(g[k].inv_tau) : 0.0f;
    }
}

__global__ void mlp_targets_kernel(int64_t n, const float *V, const float *ca, float *T) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float o[MO];
    exact_targets(V[k], ca[k], o);
    for (int j = 0; j < MO; ++j) T[k * MO + j] = o[j];
}

// per-output sums of t and t^2 (double) over a block's share of the samples
__global__ void mlp_stats_kernel(int64_t n, const float *T, double *partial) {
    __shared__ double s1[256], s2[256];
    const int o = blockIdx.y;
    double a = 0.0, b = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double t = T[k * MO + o];
        a += t;
        b += t * t;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[((int64_t)o * gridDim.x + blockIdx.x) * 2] = s1[0];
        partial[((int64_t)o * gridDim.x + blockIdx.x) * 2 + 1] = s2[0];
    }
}

// shift = mean, scale = std (>= 1e-3) per output; masked outputs keep (0, 1)
__global__ void mlp_stats_final_kernel(int64_t n, int nblocks, const double *partial, const float *mask, float *shift,
                                       float *scale) {
    const int o = threadIdx.x;
    if (o >= MO) return;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nblocks; ++i) {
        a += partial[((int64_t)o * nblocks + i) * 2];
        b += partial[((int64_t)o * nblocks + i) * 2 + 1];
    }
    const double mean = a / (double)n;
    const double var = fmax(b / (double)n - mean * mean, 0.0);
    if (mask[o] == 0.0f) {
        shift[o] = 0.0f;
        scale[o] = 1.0f;
    } else {
        shift[o] = (float)mean;
        scale[o] = (float)fmax(sqrt(var), 1e-3);
    }
}

__global__ void mlp_normalise_kernel(int64_t n, const float *V, const float *ca, float lc_mid, float lc_half,
                                     const float *shift, const float *scale, float *X, float *T) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    X[2 * k] = (V[k] - V_CENTER) / V_HALF;
    X[2 * k + 1] = (logf(ca[k]) - lc_mid) / lc_half;
    for (int j = 0; j < MO; ++j) T[k * MO + j] = (T[k * MO + j] - shift[j]) / scale[j];
}

// ---- training: one minibatch, forward + backward per sample, partial gradients per CTA ----
// Samples of the minibatch: local index j in [0, B) maps to sample (mul * (j0 + j) + add) mod n
// (a bijection when gcd(mul, n) = 1: a cheap per-epoch reshuffle).
struct GradArgs {
    const float *params;   // P_TOTAL
    const float *X;        // n x 2 normalised inputs
    const float *T;        // n x 24 normalised targets
    const float *mask;     // 24
    int64_t n;
    int64_t j0;
    int32_t B;
    uint64_t mul, add;
    float denom;           // B * sum(mask)
    float *partial;        // gridDim.x x (P_TOTAL + 1): gradient, then the loss sum
};

__global__ void __launch_bounds__(MB) mlp_grad_kernel(const GradArgs a) {
    extern __shared__ __align__(16) float sm[];
    float *Wt = sm;                          // P_TOTAL
    float *H1 = Wt + P_TOTAL;                // [MB][HS]
    float *H2 = H1 + MB * HS;
    float *D1 = H2 + MB * HS;
    float *D2 = D1 + MB * HS;
    float *D3 = D2 + MB * HS;                // [MB][MO + 1]
    float *Xs = D3 + MB * (MO + 1);          // [MB][2]
    __shared__ float red[MB];
    const int s = threadIdx.x;
    for (int p = s; p < P_TOTAL; p += MB) Wt[p] = a.params[p];
    const int64_t jl = (int64_t)blockIdx.x * MB + s;
    const bool valid = jl < a.B;
    const int64_t k = valid ? (int64_t)((a.mul * (uint64_t)(a.j0 + jl) + a.add) % (uint64_t)a.n) : 0;
    __syncthreads();
    const float *w1 = Wt + P_W1, *b1 = Wt + P_B1, *w2 = Wt + P_W2, *b2 = Wt + P_B2, *w3 = Wt + P_W3, *b3 = Wt + P_B3;
    float loss = 0.0f;
    const float x0 = valid ? a.X[2 * k] : 0.0f, x1 = valid ? a.X[2 * k + 1] : 0.0f;
    Xs[2 * s] = x0;
    Xs[2 * s + 1] = x1;
    for (int j = 0; j < MH; ++j) H1[s * HS + j] = tanhf(fmaf(w1[2 * j], x0, fmaf(w1[2 * j + 1], x1, b1[j])));
    for (int j = 0; j < MH; ++j) {
        float acc = b2[j];
        for (int q = 0; q < MH; ++q) acc = fmaf(w2[j * MH + q], H1[s * HS + q], acc);
        H2[s * HS + j] = tanhf(acc);
    }
    for (int o = 0; o < MO; ++o) {
        float acc = b3[o];
        for (int q = 0; q < MH; ++q) acc = fmaf(w3[o * MH + q], H2[s * HS + q], acc);
        const float e = valid ? (acc - a.T[k * MO + o]) * a.mask[o] : 0.0f;
        loss = fmaf(e, e, loss);
        D3[s * (MO + 1) + o] = 2.0f * e / a.denom;
    }
    for (int q = 0; q < MH; ++q) {
        float acc = 0.0f;
        for (int o = 0; o < MO; ++o) acc = fmaf(w3[o * MH + q], D3[s * (MO + 1) + o], acc);
        const float h = H2[s * HS + q];
        D2[s * HS + q] = acc * (1.0f - h * h);
    }
    for (int q = 0; q < MH; ++q) {
        float acc = 0.0f;
        for (int j = 0; j < MH; ++j) acc = fmaf(w2[j * MH + q], D2[s * HS + j], acc);
        const float h = H1[s * HS + q];
        D1[s * HS + q] = acc * (1.0f - h * h);
    }
    red[s] = loss;
    __syncthreads();
    // weight gradients of this CTA: sums over its samples, in sample order
    float *out = a.partial + (int64_t)blockIdx.x * (P_TOTAL + 1);
    {   // W2, b2: thread -> column q = s % 64, rows j in [32 (s / 64), +32)
        const int q = s % MH, jh = s / MH;
        float acc[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) acc[r] = 0.0f;
        for (int t = 0; t < MB; ++t) {
            const float h = H1[t * HS + q];
#pragma unroll
            for (int r = 0; r < 32; ++r) acc[r] = fmaf(D2[t * HS + jh * 32 + r], h, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < 32; ++r) out[P_W2 + (jh * 32 + r) * MH + q] = acc[r];
    }
    {   // W3, b3: thread -> column q, outputs o in [12 (s / 64), +12)
        const int q = s % MH, oh = s / MH;
        float acc[12];
#pragma unroll
        for (int r = 0; r < 12; ++r) acc[r] = 0.0f;
        for (int t = 0; t < MB; ++t) {
            const float h = H2[t * HS + q];
#pragma unroll
            for (int r = 0; r < 12; ++r) acc[r] = fmaf(D3[t * (MO + 1) + oh * 12 + r], h, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < 12; ++r) out[P_W3 + (oh * 12 + r) * MH + q] = acc[r];
    }
    {   // W1 (thread -> hidden unit j = s % 64, input i = s / 64), b1, b2, b3
        const int j = s % MH, i = s / MH;
        float acc = 0.0f, bacc = 0.0f, b2acc = 0.0f;
        for (int t = 0; t < MB; ++t) {
            acc = fmaf(D1[t * HS + j], Xs[2 * t + i], acc);
            bacc += D1[t * HS + j];
            b2acc += D2[t * HS + j];
        }
        out[P_W1 + j * MI + i] = acc;
        if (i == 0) out[P_B1 + j] = bacc;
        else out[P_B2 + j] = b2acc;
        if (s < MO) {
            float b3acc = 0.0f;
            for (int t = 0; t < MB; ++t) b3acc += D3[t * (MO + 1) + s];
            out[P_B3 + s] = b3acc;
        }
    }
    if (s == 0) {
        float L = 0.0f;
        for (int t = 0; t < MB; ++t) L += red[t];
        out[P_TOTAL] = L;
    }
}

size_t mlp_grad_smem() { return (size_t)(P_TOTAL + 4 * MB * HS + MB * (MO + 1) + 2 * MB) * sizeof(float); }

// Sum the CTA partials in a fixed order; then either return the gradient (grad != NULL)
// or take an Adam step on params.  Thread P_TOTAL adds the loss (divided by denom) to *loss.
__global__ void mlp_adam_kernel(const float *partial, int nblk, float *params, float *m, float *v, float *grad,
                                float lr, float b1, float b2, float eps, float c1, float c2, float denom, float *loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > P_TOTAL) return;
    float g = 0.0f;
    for (int b = 0; b < nblk; ++b) g += partial[(int64_t)b * (P_TOTAL + 1) + p];
    if (p == P_TOTAL) {
        if (loss) *loss += g / denom;
        return;
    }
    if (grad) {
        grad[p] = g;
        return;
    }
    const float mm = b1 * m[p] + (1.0f - b1) * g;
    const float vv = b2 * v[p] + (1.0f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    params[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// Glorot-uniform weights from the counter-based generator, zero biases
__global__ void mlp_init_kernel(float *params, uint64_t seed) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P_TOTAL) return;
    float a = 0.0f;
    if (p < P_B1) a = sqrtf(6.0f / (MI + MH));
    else if (p >= P_W2 && p < P_B2) a = sqrtf(6.0f / (MH + MH));
    else if (p >= P_W3 && p < P_B3) a = sqrtf(6.0f / (MH + MO));
    params[p] = a == 0.0f ? 0.0f : (float)((2.0 * sm64_uniform(sm64_mix(seed + 3), (uint64_t)p) - 1.0) * a);
}

// ---- inference on the tensor cores ---------------------------------------------------------
// Device copy of a surrogate for inference: FP32 first layer, biases and normalisation;
// BF16 64x64 and 64x24 weights with rows padded to 72 (conflict-free fragment loads).
constexpr int WS = 72;
struct MlpDev {
    float w1[MH * MI], b1[MH], b2[MH], b3[MO];
    float in_shift[MI], in_scale[MI], out_shift[MO], out_scale[MO];
    __nv_bfloat16 w2[MH * WS], w3[MO * WS];
};

__global__ void mlp_pack_kernel(const ion_surrogate_weights *w, MlpDev *d) {
    const int tid = threadIdx.x;
    for (int i = tid; i < MH * MI; i += blockDim.x) d->w1[i] = w->w1[i];
    for (int i = tid; i < MH; i += blockDim.x) {
        d->b1[i] = w->b1[i];
        d->b2[i] = w->b2[i];
    }
    for (int i = tid; i < MO; i += blockDim.x) {
        d->b3[i] = w->b3[i];
        d->out_shift[i] = w->out_shift[i];
        d->out_scale[i] = w->out_scale[i];
    }
    if (tid < MI) {
        d->in_shift[tid] = w->in_shift[tid];
        d->in_scale[tid] = w->in_scale[tid];
    }
    for (int i = tid; i < MH * WS; i += blockDim.x) {
        const int r = i / WS, c = i % WS;
        d->w2[i] = __float2bfloat16_rn(c < MH ? w->w2[r * MH + c] : 0.0f);
    }
    for (int i = tid; i < MO * WS; i += blockDim.x) {
        const int r = i / WS, c = i % WS;
        d->w3[i] = __float2bfloat16_rn(c < MH ? w->w3[r * MH + c] : 0.0f);
    }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}
__device__ __forceinline__ uint32_t tanh_bf16x2(uint32_t x) {
    uint32_t y;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One warp evaluates 16 rows (one m-tile).  in0/in1: normalised inputs of rows g and g+8
// (g = lane / 4).  y[nt][0..3]: outputs (row g: cols 8nt + 2t, +1; row g+8: same), t = lane % 4.
__device__ __forceinline__ void mlp_mtile(const MlpDev &W, float a0, float a1, float c0, float c1, float (&y)[3][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // layer 1 (FP32 FMAs) -> tanh on bf16 pairs -> A fragments of layer 2
    uint32_t A[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int cA = 16 * kk + 2 * t, cB = cA + 8;
        const float zg0 = fmaf(W.w1[2 * cA], a0, fmaf(W.w1[2 * cA + 1], a1, W.b1[cA]));
        const float zg1 = fmaf(W.w1[2 * cA + 2], a0, fmaf(W.w1[2 * cA + 3], a1, W.b1[cA + 1]));
        const float z80 = fmaf(W.w1[2 * cA], c0, fmaf(W.w1[2 * cA + 1], c1, W.b1[cA]));
        const float z81 = fmaf(W.w1[2 * cA + 2], c0, fmaf(W.w1[2 * cA + 3], c1, W.b1[cA + 1]));
        const float zg2 = fmaf(W.w1[2 * cB], a0, fmaf(W.w1[2 * cB + 1], a1, W.b1[cB]));
        const float zg3 = fmaf(W.w1[2 * cB + 2], a0, fmaf(W.w1[2 * cB + 3], a1, W.b1[cB + 1]));
        const float z82 = fmaf(W.w1[2 * cB], c0, fmaf(W.w1[2 * cB + 1], c1, W.b1[cB]));
        const float z83 = fmaf(W.w1[2 * cB + 2], c0, fmaf(W.w1[2 * cB + 3], c1, W.b1[cB + 1]));
        A[kk][0] = tanh_bf16x2(pack_bf16x2(zg0, zg1));
        A[kk][1] = tanh_bf16x2(pack_bf16x2(z80, z81));
        A[kk][2] = tanh_bf16x2(pack_bf16x2(zg2, zg3));
        A[kk][3] = tanh_bf16x2(pack_bf16x2(z82, z83));
    }
    // layer 2: 64 x 64 on the tensor cores
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float bl = W.b2[8 * nt + 2 * t], bh = W.b2[8 * nt + 2 * t + 1];
        acc[nt][0] = bl;
        acc[nt][1] = bh;
        acc[nt][2] = bl;
        acc[nt][3] = bh;
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const __nv_bfloat16 *row = W.w2 + (8 * nt + g) * WS + 16 * kk + 2 * t;
            mma_bf16(acc[nt], A[kk], *reinterpret_cast<const uint32_t *>(row),
                     *reinterpret_cast<const uint32_t *>(row + 8));
        }
    // tanh -> A fragments of layer 3 (accumulator layout = A layout of the next MMA)
    uint32_t A3[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        A3[kk][0] = tanh_bf16x2(pack_bf16x2(acc[2 * kk][0], acc[2 * kk][1]));
        A3[kk][1] = tanh_bf16x2(pack_bf16x2(acc[2 * kk][2], acc[2 * kk][3]));
        A3[kk][2] = tanh_bf16x2(pack_bf16x2(acc[2 * kk + 1][0], acc[2 * kk + 1][1]));
        A3[kk][3] = tanh_bf16x2(pack_bf16x2(acc[2 * kk + 1][2], acc[2 * kk + 1][3]));
    }
    // layer 3: 64 x 24
#pragma unroll
    for (int nt = 0; nt < 3; ++nt) {
        const int o = 8 * nt + 2 * t;
        y[nt][0] = W.b3[o];
        y[nt][1] = W.b3[o + 1];
        y[nt][2] = W.b3[o];
        y[nt][3] = W.b3[o + 1];
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int nt = 0; nt < 3; ++nt) {
            const __nv_bfloat16 *row = W.w3 + (8 * nt + g) * WS + 16 * kk + 2 * t;
            mma_bf16(y[nt], A3[kk], *reinterpret_cast<const uint32_t *>(row),
                     *reinterpret_cast<const uint32_t *>(row + 8));
        }
    // back to physical units
#pragma unroll
    for (int nt = 0; nt < 3; ++nt) {
        const int o = 8 * nt + 2 * t;
        y[nt][0] = fmaf(y[nt][0], W.out_scale[o], W.out_shift[o]);
        y[nt][1] = fmaf(y[nt][1], W.out_scale[o + 1], W.out_shift[o + 1]);
        y[nt][2] = fmaf(y[nt][2], W.out_scale[o], W.out_shift[o]);
        y[nt][3] = fmaf(y[nt][3], W.out_scale[o + 1], W.out_shift[o + 1]);
    }
}

__device__ __forceinline__ void load_mlp(MlpDev &dst, const MlpDev *src) {
    const int4 *s = reinterpret_cast<const int4 *>(src);
    int4 *d = reinterpret_cast<int4 *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(MlpDev) / 16); i += blockDim.x) d[i] = s[i];
}

// ---- the cell update with learned rates ------------------------------------------------------
// 64 threads; warp w owns CPW = 16 cells [base, base + 16): rows 0..15 dendrite (V_dend,
// [Ca]), 16..31 soma (V_soma, [Ca]), 32..47 axon (V_axon, [Ca]); three m-tiles of 16 rows.
// (16 rather than 32 cells per warp doubles the warps of a launch: the kernel is bound by
// latency, not by the tensor cores.)  Lanes 0..15 then run their cells' updates.
struct SurrArgs {
    StepCommon c;
    const MlpDev *mlp;
    const float *ic;    // gap currents of this step (NULL: none)
};

// x_inf = 1 / (1 + e^{-logit}), 1 / tau = e^{-ln tau}
__device__ __forceinline__ float learned_xinf(const float *y, int gate) {
    return rcp_approx(1.0f + ex2_approx(-y[2 * gate] * 1.4426950408889634f));
}
__device__ __forceinline__ Rate learned_rate(const float *y, int gate) {
    return Rate{learned_xinf(y, gate), ex2_approx(-y[2 * gate + 1] * 1.4426950408889634f)};
}

constexpr int SURR_CPW = 16;   // cells per warp

__global__ void __launch_bounds__(64) surrogate_cell_kernel(const SurrArgs a) {
    __shared__ __align__(16) MlpDev W;
    __shared__ float ys[2][3 * SURR_CPW][MO + 1];
    pdl_enter();
    const StepCommon &c = a.c;
    load_mlp(W, a.mlp);
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, warp = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * 2 + warp) * SURR_CPW;
    const int64_t tstep = step_index(c);
    const float *vcur = vd_cur(c);
    float *vnext = vd_next(c);
    __syncthreads();
#pragma unroll 1
    for (int mt = 0; mt < 3; ++mt) {
        const int comp = mt;                 // 0 dendrite, 1 soma, 2 axon
        const int64_t ia = base + g, ib = ia + 8;
        const float *vsrc = comp == 0 ? vcur : c.S.f(comp == 1 ? F_VSOMA : F_VAXON);
        const float va = ia < c.n ? vsrc[ia] : -60.0f, vb = ib < c.n ? vsrc[ib] : -60.0f;
        const float ca_a = ia < c.n ? c.S.f(F_CA)[ia] : 1.0f, ca_b = ib < c.n ? c.S.f(F_CA)[ib] : 1.0f;
        float y[3][4];
        mlp_mtile(W, (va - W.in_shift[0]) * W.in_scale[0], (logf(ca_a) - W.in_shift[1]) * W.in_scale[1],
                  (vb - W.in_shift[0]) * W.in_scale[0], (logf(ca_b) - W.in_shift[1]) * W.in_scale[1], y);
        const int row = comp * SURR_CPW + g;
#pragma unroll
        for (int nt = 0; nt < 3; ++nt) {
            const int o = 8 * nt + 2 * t;
            ys[warp][row][o] = y[nt][0];
            ys[warp][row][o + 1] = y[nt][1];
            ys[warp][row + 8][o] = y[nt][2];
            ys[warp][row + 8][o + 1] = y[nt][3];
        }
    }
    __syncwarp();
    const int64_t i = base + lane;
    if (lane >= SURR_CPW || i >= c.n) return;
    const Cell cell = load_cell(c.S, vcur, i);
    const float *yd = ys[warp][lane], *ysm = ys[warp][SURR_CPW + lane], *yax = ys[warp][2 * SURR_CPW + lane];
    CellRates gr;
    gr.r = learned_rate(yd, G_R);
    gr.s = learned_rate(yd, G_S);
    gr.q = learned_rate(yd, G_Q);
    gr.k = learned_rate(ysm, G_K);
    gr.l = learned_rate(ysm, G_L);
    gr.ms = Rate{learned_xinf(ysm, G_MS), 0.0f};
    gr.hs = learned_rate(ysm, G_HS);
    gr.ns = learned_rate(ysm, G_NS);
    gr.xs = learned_rate(ysm, G_XS);
    gr.ma = Rate{learned_xinf(yax, G_MA), 0.0f};
    gr.ha = learned_rate(yax, G_HA);
    gr.xa = learned_rate(yax, G_XA);
    const float ic = a.ic != nullptr ? a.ic[i] : 0.0f;
    float iapp = pulse_current(c.pulses, i, tstep);
    if (c.iapp != nullptr) iapp += c.iapp[i];
    const CellNext o = cell_step_rates(c.P, cell, ic, iapp, gr);
    finish_cell(c, tstep, vnext, i, o);
}

}  // namespace ion

using namespace ion;

// ---- host -------------------------------------------------------------------------------------
static ion_status mlp_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return ION_OK;
    return ion_fail(nullptr, ION_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static uint64_t coprime_multiplier(uint64_t n, uint64_t seed) {
    // an odd multiplier near n * 0.618..., coprime with n (a bijection of Z_n)
    auto gcd = [](uint64_t x, uint64_t y) {
        while (y) {
            const uint64_t r = x % y;
            x = y;
            y = r;
        }
        return x;
    };
    uint64_t m = (uint64_t)(0.6180339887498949 * (double)n) + 2 * (seed % 97) + 1;
    while (gcd(m, n) != 1) ++m;
    return m;
}

extern "C" ion_status ion_surrogate_train(const ion_train_cfg *cfg, ion_surrogate_weights *w_out, float *final_loss) {
    if (!cfg || !w_out) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_surrogate_train: NULL argument");
    const int64_t n = cfg->n_samples;
    const int B = cfg->batch;
    if (n < 256 || B < MB || B % MB != 0 || B > n || cfg->epochs < 1 || !(cfg->lr > 0) || !(cfg->v_hi > cfg->v_lo) ||
        !(cfg->ca_lo > 0) || !(cfg->ca_hi > cfg->ca_lo))
        return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_surrogate_train: bad configuration");
    cudaStream_t st = (cudaStream_t)cfg->cuda_stream;
    const int nblk = B / MB;
    const size_t smem = mlp_grad_smem();
    float *V = nullptr, *ca = nullptr, *X = nullptr, *T = nullptr, *params = nullptr, *m = nullptr, *v = nullptr,
          *partial = nullptr, *mask = nullptr, *shift = nullptr, *scale = nullptr, *loss = nullptr;
    double *stat = nullptr;
    const int sblk = 64;
    std::vector<void *> bufs;
    auto alloc = [&](void **p, size_t bytes) {
        cudaError_t e = ion_alloc(p, bytes);
        if (e == cudaSuccess) bufs.push_back(*p);
        return e;
    };
    auto cleanup = [&]() {
        for (void *p : bufs) cudaFree(p);
    };
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = alloc((void **)&V, n * 4);
    if (e == cudaSuccess) e = alloc((void **)&ca, n * 4);
    if (e == cudaSuccess) e = alloc((void **)&X, n * 8);
    if (e == cudaSuccess) e = alloc((void **)&T, n * MO * 4);
    if (e == cudaSuccess) e = alloc((void **)&params, P_TOTAL * 4);
    if (e == cudaSuccess) e = alloc((void **)&m, P_TOTAL * 4);
    if (e == cudaSuccess) e = alloc((void **)&v, P_TOTAL * 4);
    if (e == cudaSuccess) e = alloc((void **)&partial, (size_t)nblk * (P_TOTAL + 1) * 4);
    if (e == cudaSuccess) e = alloc((void **)&mask, MO * 4);
    if (e == cudaSuccess) e = alloc((void **)&shift, MO * 4);
    if (e == cudaSuccess) e = alloc((void **)&scale, MO * 4);
    if (e == cudaSuccess) e = alloc((void **)&loss, 4);
    if (e == cudaSuccess) e = alloc((void **)&stat, (size_t)MO * sblk * 2 * 8);
    if (e != cudaSuccess) {
        cleanup();
        return ion_fail(nullptr, ION_ERR_OOM, "ion_surrogate_train: %s", cudaGetErrorString(e));
    }
    float hmask[MO];
    for (int o = 0; o < MO; ++o) hmask[o] = (o == 2 * G_MS + 1 || o == 2 * G_MA + 1) ? 0.0f : 1.0f;
    const float lc_lo = logf(cfg->ca_lo), lc_hi = logf(cfg->ca_hi);
    const float lc_mid = 0.5f * (lc_lo + lc_hi), lc_half = 0.5f * (lc_hi - lc_lo);
    const unsigned g1 = (unsigned)((n + 255) / 256);
    e = cudaMemcpyAsync(mask, hmask, sizeof hmask, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        mlp_samples_kernel<<<g1, 256, 0, st>>>(n, cfg->seed, cfg->v_lo, cfg->v_hi, lc_lo, lc_hi, V, ca);
        mlp_targets_kernel<<<g1, 256, 0, st>>>(n, V, ca, T);
        mlp_stats_kernel<<<dim3(sblk, MO), 256, 0, st>>>(n, T, stat);
        mlp_stats_final_kernel<<<1, 32, 0, st>>>(n, sblk, stat, mask, shift, scale);
        mlp_normalise_kernel<<<g1, 256, 0, st>>>(n, V, ca, lc_mid, lc_half, shift, scale, X, T);
        mlp_init_kernel<<<(P_TOTAL + 255) / 256, 256, 0, st>>>(params, cfg->seed);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(m, 0, P_TOTAL * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, P_TOTAL * 4, st);
    const int64_t steps_per_epoch = n / B;
    const int64_t total = steps_per_epoch * cfg->epochs;
    const float denom = (float)B * 22.0f;
    int64_t step = 0;
    for (int ep = 0; ep < cfg->epochs && e == cudaSuccess; ++ep) {
        const uint64_t mul = coprime_multiplier((uint64_t)n, cfg->seed + ep);
        const uint64_t add = (uint64_t)(ep * 7919) % (uint64_t)n;
        if (ep == cfg->epochs - 1) e = cudaMemsetAsync(loss, 0, 4, st);
        for (int64_t b = 0; b < steps_per_epoch && e == cudaSuccess; ++b, ++step) {
            GradArgs ga{params, X, T, mask, n, b * B, B, mul, add, denom, partial};
            mlp_grad_kernel<<<nblk, MB, smem, st>>>(ga);
            // cosine decay of the step size to 1 % over the run
            const double frac = total > 1 ? (double)step / (double)(total - 1) : 1.0;
            const float lr = (float)(cfg->lr * (0.01 + 0.99 * 0.5 * (1.0 + cos(M_PI * frac))));
            const double k = (double)(step + 1);
            const float c1 = (float)(1.0 - pow(0.9, k)), c2 = (float)(1.0 - pow(0.999, k));
            mlp_adam_kernel<<<(P_TOTAL + 1 + 255) / 256, 256, 0, st>>>(partial, nblk, params, m, v, nullptr, lr, 0.9f,
                                                                        0.999f, 1e-8f, c1, c2, denom,
                                                                        ep == cfg->epochs - 1 ? loss : nullptr);
            e = cudaGetLastError();
        }
    }
    float hl = 0.0f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(w_out, params, P_TOTAL * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w_out->out_shift, shift, MO * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w_out->out_scale, scale, MO * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hl, loss, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "ion_surrogate_train: %s", cudaGetErrorString(e));
    // input normalisation: x' = (x - shift) * scale with x = (V, ln [Ca])
    w_out->in_shift[0] = V_CENTER;
    w_out->in_scale[0] = 1.0f / V_HALF;
    w_out->in_shift[1] = lc_mid;
    w_out->in_scale[1] = 1.0f / lc_half;
    if (final_loss) *final_loss = hl / (float)steps_per_epoch;
    return ION_OK;
}

extern "C" ion_status ion_surrogate_grad(const ion_surrogate_weights *w, const float *x, const float *t,
                                         const float *mask, int32_t B, ion_surrogate_weights *grad, float *loss) {
    if (!w || !x || !t || !mask || !grad || B < 1)
        return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_surrogate_grad: bad arguments");
    const int nblk = (B + MB - 1) / MB;
    float msum = 0.0f;
    for (int o = 0; o < MO; ++o) msum += mask[o];
    if (!(msum > 0)) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_surrogate_grad: empty mask");
    float *params = nullptr, *X = nullptr, *T = nullptr, *M = nullptr, *partial = nullptr, *g = nullptr, *L = nullptr;
    cudaError_t e = ion_alloc(&params, P_TOTAL * 4);
    if (e == cudaSuccess) e = ion_alloc(&X, (size_t)B * 8);
    if (e == cudaSuccess) e = ion_alloc(&T, (size_t)B * MO * 4);
    if (e == cudaSuccess) e = ion_alloc(&M, MO * 4);
    if (e == cudaSuccess) e = ion_alloc(&partial, (size_t)nblk * (P_TOTAL + 1) * 4);
    if (e == cudaSuccess) e = ion_alloc(&g, P_TOTAL * 4);
    if (e == cudaSuccess) e = ion_alloc(&L, 4);
    if (e == cudaSuccess) e = cudaMemcpy(params, w, P_TOTAL * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(X, x, (size_t)B * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(T, t, (size_t)B * MO * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(M, mask, MO * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(L, 0, 4);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_grad_smem());
    const float denom = (float)B * msum;
    if (e == cudaSuccess) {
        GradArgs ga{params, X, T, M, B, 0, B, 1, 0, denom, partial};
        mlp_grad_kernel<<<nblk, MB, mlp_grad_smem()>>>(ga);
        mlp_adam_kernel<<<(P_TOTAL + 1 + 255) / 256, 256>>>(partial, nblk, params, nullptr, nullptr, g, 0, 0, 0, 0, 1, 1,
                                                             denom, L);
        e = cudaGetLastError();
    }
    float hl = 0.0f;
    if (e == cudaSuccess) e = cudaMemcpy(grad, g, P_TOTAL * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hl, L, 4, cudaMemcpyDeviceToHost);
    cudaFree(params);
    cudaFree(X);
    cudaFree(T);
    cudaFree(M);
    cudaFree(partial);
    cudaFree(g);
    cudaFree(L);
    if (e != cudaSuccess)
        return ion_fail(nullptr, e == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA, "ion_surrogate_grad: %s",
                        cudaGetErrorString(e));
    if (loss) *loss = hl;
    return ION_OK;
}

// Upload a surrogate (host struct) as the packed inference copies: the warp-MMA layout
// (*d_out, may be NULL) and the tcgen05 layout (*d_tc).
ion_status ion_mlp_upload(const ion_surrogate_weights *w, void **d_out, void **d_tc, cudaStream_t st) {
    ion_surrogate_weights *dw = nullptr;
    MlpDev *d = nullptr;
    void *t = nullptr;
    cudaError_t e = ion_alloc(&dw, sizeof *dw);
    if (e == cudaSuccess && d_out) e = ion_alloc(&d, sizeof *d);
    if (e == cudaSuccess) e = ion_alloc(&t, surrogate_tc_weights_bytes());
    if (e == cudaSuccess) e = cudaMemcpyAsync(dw, w, sizeof *dw, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && d_out) {
        mlp_pack_kernel<<<1, 256, 0, st>>>(dw, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = surrogate_tc_pack(dw, t, st);
    if (e == cudaSuccess) e = surrogate_tc_prepare();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dw);
    if (e != cudaSuccess) {
        cudaFree(d);
        cudaFree(t);
        return ion_fail(nullptr, e == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA, "surrogate upload: %s",
                        cudaGetErrorString(e));
    }
    if (d_out) *d_out = d;
    *d_tc = t;
    return ION_OK;
}

extern "C" ion_status ion_surrogate_eval(const ion_surrogate_weights *w, const float *V, const float *ca, int64_t n,
                                         float *out) {
    if (!w || !V || !ca || !out || n < 1) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_surrogate_eval: bad arguments");
    void *t = nullptr;
    ion_status st = ion_mlp_upload(w, nullptr, &t, nullptr);
    if (st != ION_OK) return st;
    float *dV = nullptr, *dc = nullptr, *dout = nullptr;
    uint32_t *dstat = nullptr;
    cudaError_t e = ion_alloc(&dV, n * 4);
    if (e == cudaSuccess) e = ion_alloc(&dc, n * 4);
    if (e == cudaSuccess) e = ion_alloc(&dout, n * MO * 4);
    if (e == cudaSuccess) e = ion_alloc(&dstat, 4);
    if (e == cudaSuccess) e = cudaMemset(dstat, 0, 4);
    if (e == cudaSuccess) e = cudaMemcpy(dV, V, n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ca, n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_mlp_eval_tc(t, n, dV, dc, dout, dstat, nullptr);
    uint32_t hstat = 0;
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, n * MO * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hstat, dstat, 4, cudaMemcpyDeviceToHost);
    cudaFree(dV);
    cudaFree(dc);
    cudaFree(dout);
    cudaFree(dstat);
    cudaFree(t);
    if (e != cudaSuccess)
        return ion_fail(nullptr, e == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA, "ion_surrogate_eval: %s",
                        cudaGetErrorString(e));
    if (hstat & ST_TIMEOUT) return ion_fail(nullptr, ION_ERR_TIMEOUT, "ion_surrogate_eval: a tensor-core wait timed out");
    return ION_OK;
}

// ---- a simulation handle with learned rates -----------------------------------------------------
// Per step: the gap-junction kernel writes the currents (split mode), then the surrogate
// cell kernel runs the MLP and the update.
static cudaError_t surrogate_step(ion_sim *s, int k_off, const float *iapp) {
    const StepCommon c = ion_step_common(s, k_off, iapp);
    cudaError_t e = cudaSuccess;
    if (s->kind == ION_DENSE_UNIFORM) {
        DenseArgs a{};
        a.c = c;
        a.g = s->g;
        a.kahan = 1;
        a.fuse = 0;
        a.ic_out = s->d_ic;
        e = launch_dense_step(a, s->dense_R, s->dense_W, s->dense_GJ, s->st);
        s->launches++;
    } else if (s->kind == ION_CSR) {
        CsrArgs a{};
        a.c = c;
        ion_csr_fill(s, a, false);
        a.fuse = 0;
        a.ic_out = s->d_ic;
        e = launch_csr_step(a, s->csr_SW, s->csr_rows, s->st);
        s->launches++;
    }
    if (e != cudaSuccess) return e;
    s->launches++;
    const float *ic = s->kind == ION_NO_GJ ? nullptr : s->d_ic;
    if (!(s->flags & ION_FLAG_SURROGATE_WARP_MMA)) return launch_surrogate_tc(c, s->d_mlp_tc, ic, s->st);
    SurrArgs sa{c, (const MlpDev *)s->d_mlp, ic};
    return launch_k(surrogate_cell_kernel, dim3((unsigned)((s->n + 2 * SURR_CPW - 1) / (2 * SURR_CPW))), dim3(64), 0,
                    s->st, c.pdl != 0, sa);
}

ion_status ion_setup_surrogate(ion_sim *s, const ion_params *p) {
    if (!p->surrogate) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "surrogate: no weights");
    ion_status st = ion_mlp_upload((const ion_surrogate_weights *)p->surrogate, &s->d_mlp, &s->d_mlp_tc, s->st);
    if (st != ION_OK) return st;
    if (s->kind != ION_NO_GJ && !s->d_ic) {
        cudaError_t e = ion_alloc(&s->d_ic, (size_t)s->n_pad * sizeof(float));
        if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_OOM, "surrogate: %s", cudaGetErrorString(e));
    }
    s->step_override = surrogate_step;
    s->lps = s->kind == ION_NO_GJ ? 1 : 2;
    s->csr_staged = 0;
    return ION_OK;
}
