// ion_mlp_tc.cu -- inference of the learned rate-function surrogate (not in the paper) on
// the fifth-generation tensor cores: tcgen05.mma with TMEM accumulators.
//
// The surrogate is the MLP of ion_mlp.cu: (V, ln[Ca]) -> 64 tanh -> 64 tanh -> 24 outputs
// (logit x_inf and ln tau of every gate).  A CTA of 128 threads owns 128 cells and
// evaluates the MLP for their three compartments (V_dend, V_soma, V_axon, each with the
// cell's [Ca]) as three 128-row tiles: row t of every tile is cell t of the CTA, so thread
// t ends up holding all three compartments' rates and runs that cell's explicit-Euler
// update itself.  The tiles go through the two layers one after the other (a version
// that pushed all three through each layer together, two tensor-core waits per step
// instead of six, measured slower: it needs twice the TMEM and shared memory per CTA, so
// half as many CTAs share an SM):
//   layer 1 (2 -> 64) in FP32 on the CUDA cores, tanh on packed bf16 pairs, written to
//     shared memory as the three BF16 A operands of layer 2;
//   layer 2 (64 x 64): four tcgen05.mma.kind::f16 (M = 128, N = 64, K = 16 each, BF16 in,
//     FP32 accumulation) into TMEM columns 0..63, issued by one thread and completed
//     through one tcgen05.commit on an mbarrier;
//   every thread reads its row of each tile back (tcgen05.ld, lane = row), adds the bias,
//     applies tanh and writes the tile's BF16 A operand of layer 3 over its layer-2 one;
//   layer 3 (64 x 24, padded to N = 32): four MMAs into TMEM columns 0..31 (over the
//     layer-2 results, already read), one commit, read back and mapped to physical units.
// Operands use the canonical K-major layout without swizzling: 8-row x 16-byte core
// matrices of 128 contiguous bytes, core matrix (row group g, K chunk c) at byte
// (8 g + c) 128, so the K-direction core-matrix stride (leading byte offset) is 128 B and
// the row-group stride (stride byte offset) 1024 B.
// Every wait is bounded: a tensor-core completion that does not arrive within ~0.5 s sets
// the timeout status bit; the CTA then waits (again bounded) once more, frees its TMEM and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ion.h"
#include "ion_kernels.cuh"
#include "ion_sim.h"

namespace ion {
namespace tc {

constexpr int ROWS = 128;        // M of every MMA: rows (cells) per CTA
constexpr int KH = 64;           // hidden width (K of layers 2 and 3)
constexpr int N2 = 64, N3 = 32;  // layer 2 outputs; layer 3 outputs (24) padded to a multiple of 16
constexpr int NOUT = ION_MLP_OUT;
constexpr int NT = 1;                 // tiles through a layer at once (see above)
constexpr uint32_t TMEM_COLS = 128;   // layer 2: tile c in [64 c, 64 c + 64); layer 3: [32 c, 32 c + 32)
constexpr float LOG2E = 1.4426950408889634f;

__host__ __device__ constexpr int core_off(int row, int kchunk) {
    return ((row >> 3) * (KH / 8) + kchunk) * 128 + (row & 7) * 16;
}

// Weights as the kernels use them (packed once per handle by mlp_tc_pack_kernel).
struct Weights {
    __nv_bfloat16 w2[N2 * KH];   // B of layer 2 (row = output unit), core-matrix layout
    __nv_bfloat16 w3[N3 * KH];   // B of layer 3, rows 24..31 zero
    float w1[2 * KH], b1[KH], b2[N2], b3[N3];
    float in_shift[2], in_scale[2], out_shift[N3], out_scale[N3];
};
struct Smem {
    __nv_bfloat16 a[NT][ROWS * KH];   // A of layer 2, then of layer 3, per tile
    Weights W;
    uint64_t bar;
    uint32_t tmem;
    int ok;
};
static_assert(sizeof(Weights) % 16 == 0, "weights are copied 16 bytes at a time");
static_assert(offsetof(Smem, W) % 16 == 0, "16-byte aligned operands");

// ---- tcgen05 / TMEM primitives (inline PTX) ------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// D[tmem] (+)= A[smem] x B[smem]^T, both K-major; accumulate = 0 overwrites D
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive once on `bar` when every MMA this thread issued before has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 32 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading (K-direction) and stride
// (row-group) byte offsets, descriptor version 1, no swizzling.
__device__ __forceinline__ uint64_t smem_desc(const void *p, uint32_t lbo, uint32_t sbo) {
    const uint32_t a = smem_u32(p);
    return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
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

// Issue one layer for `tiles` tiles (four K = 16 steps each; tile c's accumulator at TMEM
// column d_tmem + c * d_stride) from thread 0 and wait for it in every thread.  Returns
// false (in every thread) if the completion did not arrive in time.
__device__ __forceinline__ bool tc_layer(Smem &sm, int tiles, const __nv_bfloat16 *B, uint32_t d_tmem,
                                         uint32_t d_stride, uint32_t idesc, uint32_t &phase) {
    if (threadIdx.x == 0) {
        tc_fence_after();
        for (int c = 0; c < tiles; ++c)
#pragma unroll
            for (int kk = 0; kk < KH / 16; ++kk)
                tc_mma(d_tmem + c * d_stride, smem_desc(sm.a[c] + kk * 16 * 8, 128, 1024),
                       smem_desc(B + kk * 16 * 8, 128, 1024), idesc, kk > 0 ? 1u : 0u);
        tc_commit(&sm.bar);
    }
    const bool done = mbar_wait_bounded(&sm.bar, phase & 1u);
    phase++;
    tc_fence_after();
    return !__syncthreads_or(!done);
}

// Layer 1 of one row of tile c: z = W1 x + b1 (FP32), tanh on bf16 pairs, into A (core-matrix layout).
__device__ __forceinline__ void layer1_row(Smem &sm, int c, int row, float x0, float x1) {
    char *abase = reinterpret_cast<char *>(sm.a[c]);
#pragma unroll
    for (int kc = 0; kc < KH / 8; ++kc) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int j = 8 * kc + 2 * h;
            const float z0 = fmaf(sm.W.w1[2 * j], x0, fmaf(sm.W.w1[2 * j + 1], x1, sm.W.b1[j]));
            const float z1 = fmaf(sm.W.w1[2 * j + 2], x0, fmaf(sm.W.w1[2 * j + 3], x1, sm.W.b1[j + 1]));
            w[h] = tanh_bf16x2(pack_bf16x2(z0, z1));
        }
        *reinterpret_cast<uint4 *>(abase + core_off(row, kc)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Layer-2 epilogue of this thread's row of tile c: + b2, tanh, into the tile's A operand
// of layer 3 (over its layer-2 operand, which the completed MMAs no longer read).
__device__ __forceinline__ void layer2_epilogue(Smem &sm, int c, uint32_t lane_addr, int row) {
    char *abase = reinterpret_cast<char *>(sm.a[c]);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float v[32];
        tc_ld32(lane_addr + 32 * half, v);
        tc_wait_ld();
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int j = 8 * kc + 2 * h;
                w[h] = tanh_bf16x2(pack_bf16x2(v[j] + sm.W.b2[32 * half + j], v[j + 1] + sm.W.b2[32 * half + j + 1]));
            }
            *reinterpret_cast<uint4 *>(abase + core_off(row, 4 * half + kc)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// CTA prologue: weights into shared memory, mbarrier, TMEM columns (warp 0).
__device__ __forceinline__ void tc_setup(Smem &sm, const Weights *Wg) {
    const int4 *s = reinterpret_cast<const int4 *>(Wg);
    int4 *d = reinterpret_cast<int4 *>(&sm.W);
    for (int i = threadIdx.x; i < (int)(sizeof(Weights) / 16); i += blockDim.x) d[i] = s[i];
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar, 1);
        fence_mbar_init();
    }
    if (threadIdx.x < 32) {
        tmem_alloc(&sm.tmem, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}
__device__ __forceinline__ void tc_teardown(Smem &sm) {
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(sm.tmem, TMEM_COLS);
}

// Both MMA layers for `tiles` 128-row tiles with inputs (x0[c], x1) of this thread's row;
// y[c] receives the 24 outputs of tile c in physical units.  Returns false if a completion
// timed out (status bit set).
__device__ __forceinline__ bool mlp_tiles(Smem &sm, int tiles, const float (&x0)[NT], float x1, uint32_t &phase,
                                          float (&y)[NT][NOUT], uint32_t *status) {
    const int row = threadIdx.x;
    const uint32_t lane_addr = sm.tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16);
    for (int c = 0; c < tiles; ++c) layer1_row(sm, c, row, x0[c], x1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    bool ok = tc_layer(sm, tiles, sm.W.w2, sm.tmem, N2, idesc_bf16(ROWS, N2), phase);
    if (ok) {
        for (int c = 0; c < tiles; ++c) layer2_epilogue(sm, c, lane_addr + c * N2, row);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        ok = tc_layer(sm, tiles, sm.W.w3, sm.tmem, N3, idesc_bf16(ROWS, N3), phase);
    }
    if (!ok) {
        if (threadIdx.x == 0 && status != nullptr) atomicOr(status, (uint32_t)ST_TIMEOUT);
        if (threadIdx.x == 0) (void)mbar_wait_bounded(&sm.bar, (phase - 1u) & 1u);   // the late MMAs, once more
        return false;
    }
    for (int c = 0; c < tiles; ++c) {
        float v[32];
        tc_ld32(lane_addr + c * N3, v);
        tc_wait_ld();
#pragma unroll
        for (int o = 0; o < NOUT; ++o) y[c][o] = fmaf(v[o] + sm.W.b3[o], sm.W.out_scale[o], sm.W.out_shift[o]);
    }
    return true;
}

__device__ __forceinline__ float learned_xinf(const float (&y)[NOUT], int gate) {
    return rcp_approx(1.0f + ex2_approx(-y[2 * gate] * LOG2E));
}
__device__ __forceinline__ Rate learned_rate(const float (&y)[NOUT], int gate) {
    return Rate{learned_xinf(y, gate), ex2_approx(-y[2 * gate + 1] * LOG2E)};
}

}  // namespace tc

struct SurrTcArgs {
    StepCommon c;
    const tc::Weights *W;
    const float *ic;    // gap currents of this step (NULL: none)
};

// The cell update with learned rates: 128 cells per CTA, three tensor-core tiles.
__global__ void __launch_bounds__(128) surrogate_tc_kernel(const SurrTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    tc::Smem &sm = *reinterpret_cast<tc::Smem *>(smem_raw);
    tc::tc_setup(sm, a.W);   // weights and TMEM are not step data: before the dependency wait
    pdl_enter();
    const StepCommon &c = a.c;
    const int64_t i = (int64_t)blockIdx.x * tc::ROWS + threadIdx.x;
    const bool valid = i < c.n;
    const int64_t tstep = step_index(c);
    const float *vcur = vd_cur(c);
    float *vnext = vd_next(c);
    Cell cell{};
    if (valid) cell = load_cell(c.S, vcur, i);
    const float ca = valid ? cell.ca : 1.0f;
    const float x1 = (logf(ca) - sm.W.in_shift[1]) * sm.W.in_scale[1];
    CellRates gr;
    uint32_t phase = 0;
    bool ok = true;
#pragma unroll 1
    for (int comp = 0; comp < 3 && ok; ++comp) {
        const float V = !valid ? -60.0f : (comp == 0 ? cell.vd : (comp == 1 ? cell.vs : cell.va));
        const float x0[tc::NT] = {(V - sm.W.in_shift[0]) * sm.W.in_scale[0]};
        float y[tc::NT][tc::NOUT];
        ok = tc::mlp_tiles(sm, 1, x0, x1, phase, y, c.status);
        if (comp == 0) {
            gr.r = tc::learned_rate(y[0], G_R);
            gr.s = tc::learned_rate(y[0], G_S);
            gr.q = tc::learned_rate(y[0], G_Q);
        } else if (comp == 1) {
            gr.k = tc::learned_rate(y[0], G_K);
            gr.l = tc::learned_rate(y[0], G_L);
            gr.ms = Rate{tc::learned_xinf(y[0], G_MS), 0.0f};
            gr.hs = tc::learned_rate(y[0], G_HS);
            gr.ns = tc::learned_rate(y[0], G_NS);
            gr.xs = tc::learned_rate(y[0], G_XS);
        } else {
            gr.ma = Rate{tc::learned_xinf(y[0], G_MA), 0.0f};
            gr.ha = tc::learned_rate(y[0], G_HA);
            gr.xa = tc::learned_rate(y[0], G_XA);
        }
    }
    tc::tc_teardown(sm);
    if (!ok || !valid) return;
    const float ic = a.ic != nullptr ? a.ic[i] : 0.0f;
    float iapp = pulse_current(c.pulses, i, tstep);
    if (c.iapp != nullptr) iapp += c.iapp[i];
    const CellNext o = cell_step_rates(c.P, cell, ic, iapp, gr);
    finish_cell(c, tstep, vnext, i, o);
}

// Batched evaluation: out[k * 24 + o] for n (V, [Ca]) pairs, 128 per CTA.
__global__ void __launch_bounds__(128) mlp_eval_tc_kernel(const tc::Weights *Wg, int64_t n, const float *V,
                                                          const float *ca, float *out, uint32_t *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    tc::Smem &sm = *reinterpret_cast<tc::Smem *>(smem_raw);
    tc::tc_setup(sm, Wg);
    const int64_t k = (int64_t)blockIdx.x * tc::ROWS + threadIdx.x;
    const bool valid = k < n;
    float x0[tc::NT] = {valid ? (V[k] - sm.W.in_shift[0]) * sm.W.in_scale[0] : 0.0f};
    const float x1 = valid ? (logf(ca[k]) - sm.W.in_shift[1]) * sm.W.in_scale[1] : 0.0f;
    uint32_t phase = 0;
    float y[tc::NT][tc::NOUT];
    const bool ok = tc::mlp_tiles(sm, 1, x0, x1, phase, y, status);
    tc::tc_teardown(sm);
    if (!ok || !valid) return;
#pragma unroll
    for (int o = 0; o < tc::NOUT; ++o) out[k * tc::NOUT + o] = y[0][o];
}

// Pack a host-layout surrogate (ion_surrogate_weights, FP32, row-major [out][in]) into the
// kernels' layout: BF16 layer-2/3 weights in core-matrix order, the rest FP32.
__global__ void mlp_tc_pack_kernel(const ion_surrogate_weights *w, tc::Weights *d) {
    for (int i = threadIdx.x; i < tc::N2 * tc::KH; i += blockDim.x) {
        const int r = i / tc::KH, k = i % tc::KH;
        d->w2[tc::core_off(r, k / 8) / 2 + (k % 8)] = __float2bfloat16_rn(w->w2[r * tc::KH + k]);
    }
    for (int i = threadIdx.x; i < tc::N3 * tc::KH; i += blockDim.x) {
        const int r = i / tc::KH, k = i % tc::KH;
        d->w3[tc::core_off(r, k / 8) / 2 + (k % 8)] = __float2bfloat16_rn(r < tc::NOUT ? w->w3[r * tc::KH + k] : 0.0f);
    }
    for (int i = threadIdx.x; i < 2 * tc::KH; i += blockDim.x) d->w1[i] = w->w1[i];
    for (int i = threadIdx.x; i < tc::KH; i += blockDim.x) {
        d->b1[i] = w->b1[i];
        d->b2[i] = w->b2[i];
    }
    for (int i = threadIdx.x; i < tc::N3; i += blockDim.x) {
        const bool real = i < tc::NOUT;
        d->b3[i] = real ? w->b3[i] : 0.0f;
        d->out_shift[i] = real ? w->out_shift[i] : 0.0f;
        d->out_scale[i] = real ? w->out_scale[i] : 0.0f;
    }
    if (threadIdx.x < 2) {
        d->in_shift[threadIdx.x] = w->in_shift[threadIdx.x];
        d->in_scale[threadIdx.x] = w->in_scale[threadIdx.x];
    }
}

// Shared memory requested per CTA: at least 56 KB, so that at most four CTAs share an SM
// and their TMEM allocations (128 of the SM's 512 columns each) never have to wait.
static constexpr size_t kTcSmem = sizeof(tc::Smem) > 56 * 1024 ? sizeof(tc::Smem) : 56 * 1024;
size_t surrogate_tc_smem() { return kTcSmem; }
size_t surrogate_tc_weights_bytes() { return sizeof(tc::Weights); }

cudaError_t surrogate_tc_prepare() {
    cudaError_t e = cudaFuncSetAttribute(surrogate_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mlp_eval_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    return e;
}

cudaError_t surrogate_tc_pack(const ion_surrogate_weights *d_w, void *d_out, cudaStream_t st) {
    mlp_tc_pack_kernel<<<1, 256, 0, st>>>(d_w, static_cast<tc::Weights *>(d_out));
    return cudaGetLastError();
}

cudaError_t launch_surrogate_tc(const StepCommon &c, const void *W, const float *ic, cudaStream_t st) {
    SurrTcArgs a{c, static_cast<const tc::Weights *>(W), ic};
    return launch_k(surrogate_tc_kernel, dim3((unsigned)((c.n + tc::ROWS - 1) / tc::ROWS)), dim3(tc::ROWS), kTcSmem,
                    st, c.pdl != 0, a);
}

cudaError_t launch_mlp_eval_tc(const void *W, int64_t n, const float *V, const float *ca, float *out,
                               uint32_t *status, cudaStream_t st) {
    mlp_eval_tc_kernel<<<(unsigned)((n + tc::ROWS - 1) / tc::ROWS), tc::ROWS, kTcSmem, st>>>(
        static_cast<const tc::Weights *>(W), n, V, ca, out, status);
    return cudaGetLastError();
}

}  // namespace ion
