// ion_dense.cu -- dense all-to-all gap-junction step (Algorithm 1 with C = 100 %), one
// launch per step or one persistent launch for many steps.
//
// For a uniform pair weight g the gap current of cell i is
//   Ic_i = g sum_j (0.8 e^{-dV_ij^2/100} + 0.2) dV_ij,  dV_ij = V_i - V_j   (j = 0..N-1).
// With m a per-step shift (V_dend of cell 0) and u = s (V - m), s = sqrt(log2(e)/100),
// the exponential is 2^{-(u_i-u_j)^2} (one SFU ex2) and the linear part sums in closed
// form, sum_j dV_ij = (N u_i - sum_j u_j) / s.  So
//   Ic_i = (g/s) [0.8 sum_j 2^{-du^2} du + 0.2 (N u_i - sum_j u_j)],  du = u_i - u_j.
// The shift keeps the rounding error of du proportional to |V - m| rather than |V|, so
// nearly synchronous cells keep their relative accuracy.
//
// Layout (N-body style): V_dend(t) is staged into shared memory in tiles of TJ floats by
// 1-D bulk async copies (cp.async.bulk, completion on an mbarrier), double-buffered when
// N > TJ.  A CTA has GR x GJ warps: GR row groups of R rows and GJ interleaved column
// splits.  Each lane holds u_i of its R rows and walks its columns four at a time: one
// 16-byte shared load of raw V_dend, centred, scaled and negated in registers
// (x_j = -(V_j - m) s: two packed f32x2 operations per four columns), then 4 x R pairs
// through packed f32x2 arithmetic (per two pairs: one FADD2, one FMUL2, two ex2, one
// FFMA2).  Lane sums are folded into Kahan-compensated accumulators every 64 columns, then
// summed pairwise across lanes (a fixed butterfly) and across column splits, so results
// are deterministic.  After the pairs every thread adds up an even share of the tile's
// x_j for the linear part's sum_j u_j.
//
// The fused step then runs the explicit-Euler cell update of the CTA's rows, one thread
// per row, from the rows' state words that cp.async copied into shared memory while the
// pair loop ran; it writes V_dend(t+1) to the other V_dend buffer.
//
// Per-step launches are programmatically dependent (launch_k, pdl_enter): the kernel may
// be scheduled while the previous step drains, initialises its mbarriers, then waits for
// that step's completion before its first global access.  The V_dend slot comes from the
// host-passed parity, so the tile copy is issued without waiting on the step counter.
#include <cuda_runtime.h>

#include "ion_async.cuh"
#include "ion_dense_core.cuh"
#include "ion_kernels.cuh"

namespace ion {

// ---- one launch per step ----------------------------------------------------------------
// Launch bounds: up to 1024 threads (64 registers) when R <= 4, else 768.
template <int R>
struct DenseBounds {
    static constexpr int threads = R <= 4 ? 1024 : 768;
};

template <int R, int GJ>
__global__ void __launch_bounds__(DenseBounds<R>::threads) dense_step_kernel(const DenseArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float red_s[32], red_c[32];
    __shared__ float U_sh;

    const StepCommon &c = a.c;
    const int n = c.n;
    const int W = blockDim.x >> 5;
    const int GR = W / GJ;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rg = warp % GR, csp = warp / GR;
    const int rows_cta = GR * R;
    const DenseSmem sm = dense_smem(smem_raw, c.n_pad);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    pdl_enter();

    const int64_t t = step_index(c);
    const float *vcur = a.vd_in != nullptr ? a.vd_in : vd_cur(c);
    float *vnext = a.fuse ? vd_next(c) : nullptr;
    const int row_base = blockIdx.x * rows_cta;
    float *cs = sm.part + W * R;              // staged Cell words of the CTA's rows
    float *ic_s = cs + NCW * rows_cta;        // their gap currents
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < 2 && k < sm.n_tiles; ++k) issue_tile(sm, vcur, c.n_pad, k, bar);
    // the rows' state words travel to shared memory while the pair loop runs
    if (a.fuse) stage_cells(cs, c.S, vcur, row_base, rows_cta, n);
    const float m_shift = vcur[0];

    float ui[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = row_base + rg * R + r;
        ui[r] = (i < n) ? (vcur[i] - m_shift) * GJ_SCALE : 0.0f;
    }
    uint32_t uses[2] = {0u, 0u};
    float tot[R], Us, Uc;
    if (!gj_pass<R, GJ>(sm, vcur, n, c.n_pad, bar, uses, m_shift, ui, csp, lane, a.kahan, tot, Us, Uc)) {
        if (threadIdx.x == 0) {
            if (c.status != nullptr) atomicOr(c.status, (uint32_t)ST_TIMEOUT);   // primitives pass none
            // let any copy still in flight land before the CTA's shared memory is released
            for (int k = 0; k < 2 && k < sm.n_tiles; ++k) (void)mbar_wait_bounded(&bar[k], uses[k] & 1u);
        }
        // the stand-alone primitive has no status word: its caller sees NaN in these rows
        if (!a.fuse)
            for (int rr = threadIdx.x; rr < rows_cta && row_base + rr < n; rr += blockDim.x)
                a.ic_out[row_base + rr] = __int_as_float(0x7fc00000);
        cp_async_wait_all();   // no staging copy may still be landing when the CTA exits
        return;
    }
    const float U = gj_reduce<R, GJ>(sm, tot, Us, Uc, rg, csp, lane, red_s, red_c, &U_sh);

    for (int rr = threadIdx.x; rr < rows_cta; rr += blockDim.x) {
        const int i = row_base + rr;
        if (i >= n) break;
        const float ic = row_current<GJ>(sm, rr, (vcur[i] - m_shift) * GJ_SCALE, n, U, a.g);
        if (!a.fuse) a.ic_out[i] = ic;
        else ic_s[rr] = ic;
    }
    if (!a.fuse) return;
    cp_async_wait_all();
    __syncthreads();
    // one thread per cell, from the staged words (ten threads per cell, cell_step_role,
    // measured slower here: 0.89 against 0.70 us per step at 8192 cells)
    for (int rr = threadIdx.x; rr < rows_cta; rr += blockDim.x) {
        const int i = row_base + rr;
        if (i >= n) break;
        float iapp = pulse_current(c.pulses, i, t);
        if (c.iapp != nullptr) iapp += c.iapp[i];
        const CellNext o = cell_step(c.P, staged_cell(cs, rows_cta, rr), ic_s[rr], iapp);
        finish_cell(c, t, vnext, i, o);
    }
}

// ---- persistent: many steps in one cooperative launch ------------------------------------
// The CTA keeps its rows' state in shared memory across steps (loaded at the start,
// written back at the end); every step stages V_dend(t) and runs the pair pass, then
// updates its rows from the shared copy: NROLE threads per cell when that fits one round
// of the CTA's threads (each thread reads its cell, then a CTA barrier, then writes), else
// one thread per cell.  V_dend(t+1) of the rows goes to the other global V_dend buffer and
// the CTAs meet at a bounded grid barrier (a release flag, grid_barrier_flag) before
// staging it for the next step.  With a single CTA and a single tile (small networks)
// V_dend never leaves shared memory: the tile is updated in place.
// Launch bounds of the persistent variant: 896 threads when R <= 4, else 576.
template <int R>
struct PersistBounds {
    static constexpr int threads = R <= 4 ? 896 : 576;
};

template <int R, int GJ>
__global__ void __launch_bounds__(PersistBounds<R>::threads) dense_persist_kernel(const PersistArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float red_s[32], red_c[32];
    __shared__ float U_sh, m_sh;
    __shared__ int ok_sh;

    const StepCommon &c = a.c;
    const int n = c.n;
    const int W = blockDim.x >> 5;
    const int GR = W / GJ;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rg = warp % GR, csp = warp / GR;
    const int rows_cta = GR * R;
    const DenseSmem sm = dense_smem(smem_raw, c.n_pad);
    float *cs = sm.part + W * R;              // the rows' 15 Cell words
    float *xs = cs + NCW * rows_cta;          // their m_s, m_a, I_CaH, I_c
    float *ic_s = xs + 4 * rows_cta;          // their gap currents
    const RoleOutSmem out{cs, xs, rows_cta};
    const bool single = gridDim.x == 1 && sm.n_tiles == 1;
    const int row_base = blockIdx.x * rows_cta;
    const int rows_here = max(0, min(rows_cta, n - row_base));
    const int64_t t0 = *c.t_dev;
    const int rows32 = (rows_cta + 31) & ~31;
    const bool roles = NROLE * rows32 <= (int)blockDim.x;

    // the rows' state from global memory
    for (int q = threadIdx.x; q < NCW * rows_cta; q += blockDim.x) {
        const int w = q / rows_cta, rr = q - w * rows_cta;
        if (rr < rows_here)
            cs[q] = w == 0 ? vd_slot(c.S, t0)[row_base + rr] : c.S.f(cell_word_field(w))[row_base + rr];
    }
    for (int q = threadIdx.x; q < 4 * rows_cta; q += blockDim.x) {
        const int k = q / rows_cta, rr = q - k * rows_cta;
        const int f = k == 0 ? F_MS : (k == 1 ? F_MA : (k == 2 ? F_ICAH : F_IC));
        if (rr < rows_here) xs[q] = c.S.f(f)[row_base + rr];
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t uses[2] = {0u, 0u};
    if (single && threadIdx.x == 0) issue_tile(sm, vd_slot(c.S, t0), c.n_pad, 0, bar);
    if (single) {   // wait for the one initial copy; afterwards the tile is updated in place
        const bool landed = mbar_wait_bounded(&bar[0], 0u);
        uses[0] = 1;
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) atomicOr(c.status, (uint32_t)ST_TIMEOUT);
            return;
        }
    }
    if (a.debug_delay_ns > 0 && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        const uint64_t d0 = globaltimer_ns();
        while (globaltimer_ns() - d0 < (uint64_t)a.debug_delay_ns) __nanosleep(1000);
    }

    int done = 0;   // steps whose update is in the shared copy
    for (int k = 0; k < a.n_steps; ++k) {
        const int64_t t = t0 + k;
        const float *vcur = vd_slot(c.S, t);
        float *vnext = vd_slot(c.S, t + 1);
        if (!single && threadIdx.x == 0)
            for (int q = 0; q < 2 && q < sm.n_tiles; ++q) issue_tile(sm, vcur, c.n_pad, q, bar);
        // shift m = V_dend of cell 0 at step t (from L2, or from the tile itself)
        if (threadIdx.x == 0) m_sh = single ? sm.tile0[0] : __ldcg(vcur);
        __syncthreads();
        const float m_shift = m_sh;
        float ui[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int rr = rg * R + r;
            ui[r] = (rr < rows_here) ? (cs[rr] - m_shift) * GJ_SCALE : 0.0f;
        }
        float tot[R], Us, Uc;
        if (!gj_pass<R, GJ>(sm, single ? nullptr : vcur, n, c.n_pad, bar, uses, m_shift, ui, csp, lane, a.kahan, tot,
                            Us, Uc)) {
            if (threadIdx.x == 0) {
                atomicOr(c.status, (uint32_t)ST_TIMEOUT);
                atomicExch(a.abort_flag, 1u);
                for (int q = 0; q < 2 && q < sm.n_tiles; ++q) (void)mbar_wait_bounded(&bar[q], uses[q] & 1u);
            }
            break;
        }
        const float U = gj_reduce<R, GJ>(sm, tot, Us, Uc, rg, csp, lane, red_s, red_c, &U_sh);
        for (int rr = threadIdx.x; rr < rows_here; rr += blockDim.x)
            ic_s[rr] = row_current<GJ>(sm, rr, (cs[rr] - m_shift) * GJ_SCALE, n, U, a.g);
        __syncthreads();
        if (roles) {   // one round: read the cell, barrier, write its new words
            const int role = threadIdx.x / rows32, rr = threadIdx.x - role * rows32;
            const bool mine = role < NROLE && rr < rows_here;
            Cell cell{};
            float iapp = 0.0f, ic = 0.0f;
            const int64_t i = row_base + rr;
            if (mine) {
                cell = staged_cell(cs, rows_cta, rr);
                ic = ic_s[rr];
                if (role == 0) {
                    iapp = pulse_current(c.pulses, i, t);
                    if (c.iapp != nullptr) iapp += c.iapp[i];
                }
            }
            __syncthreads();
            if (mine) cell_step_role(role, c, t, vnext, i, rr, cell, ic, iapp, out);
        } else {
            for (int rr = threadIdx.x; rr < rows_here; rr += blockDim.x) {
                const int64_t i = row_base + rr;
                float iapp = pulse_current(c.pulses, i, t);
                if (c.iapp != nullptr) iapp += c.iapp[i];
                const CellNext o = cell_step(c.P, staged_cell(cs, rows_cta, rr), ic_s[rr], iapp);
                put_cell_smem(out, rr, o);
                vnext[i] = o.vd;
                if (!cell_finite(o)) atomicOr(c.status, (uint32_t)ST_NONFINITE);
                if (c.trace != nullptr && ((t + 1) % c.trace_stride) == 0) {
                    const int64_t sample = (t + 1) / c.trace_stride - 1;
                    c.trace[(sample % c.trace_cap) * (int64_t)n + i] = o.va;
                }
            }
        }
        done = k + 1;
        if (single) {
            __syncthreads();                          // all pair loops are done with the tile
            for (int rr = threadIdx.x; rr < rows_here; rr += blockDim.x) sm.tile0[rr] = cs[rr];
            __syncthreads();
        } else if (!grid_barrier_flag(a.bar_count, a.bar_flag, a.abort_flag, a.bar_base + (uint32_t)(k + 1) * gridDim.x,
                                      a.timeout_ns, c.status, &ok_sh)) {
            break;
        }
    }
    // write the state back (after an aborted run: the CTA's last completed step)
    __syncthreads();
    float *vfin = vd_slot(c.S, t0 + done);
    for (int q = threadIdx.x; q < NCW * rows_cta; q += blockDim.x) {
        const int w = q / rows_cta, rr = q - w * rows_cta;
        if (rr < rows_here && w != NCW - 1) (w == 0 ? vfin : c.S.f(cell_word_field(w)))[row_base + rr] = cs[q];
    }
    for (int q = threadIdx.x; q < 4 * rows_cta; q += blockDim.x) {
        const int kk = q / rows_cta, rr = q - kk * rows_cta;
        const int f = kk == 0 ? F_MS : (kk == 1 ? F_MA : (kk == 2 ? F_ICAH : F_IC));
        if (rr < rows_here) c.S.f(f)[row_base + rr] = xs[q];
    }
}

size_t dense_smem_bytes(int n_pad, int R, int W) {
    const int n_tiles = (n_pad + TJ - 1) / TJ;
    const size_t tiles = (n_tiles > 1 ? 2 * TJ : n_pad) * sizeof(float);
    return tiles + (size_t)W * R * sizeof(float);   // part[rows_cta][GJ] = (W / GJ) * R * GJ floats
}
// the per-step kernel also stages its rows' Cell words and keeps their currents
static size_t dense_step_smem_bytes(int n_pad, int R, int W, int GJ) {
    return dense_smem_bytes(n_pad, R, W) + (size_t)(NCW + 1) * (W / GJ) * R * sizeof(float);
}

// ---- launch-shape dispatch: R rows per warp, W warps = (W / GJ) row groups x GJ splits ----
template <template <int, int> class Op, int R>
static cudaError_t dispatch_gj(int GJ, typename Op<R, 1>::Args &args) {
    switch (GJ) {
        case 1: return Op<R, 1>::run(args);
        case 2: return Op<R, 2>::run(args);
        case 4: return Op<R, 4>::run(args);
        default: return cudaErrorInvalidValue;
    }
}
template <template <int, int> class Op>
static cudaError_t dispatch(int R, int GJ, typename Op<1, 1>::Args &args) {
    switch (R) {
        case 1: return dispatch_gj<Op, 1>(GJ, args);
        case 2: return dispatch_gj<Op, 2>(GJ, args);
        case 4: return dispatch_gj<Op, 4>(GJ, args);
        case 6: return dispatch_gj<Op, 6>(GJ, args);
        case 8: return dispatch_gj<Op, 8>(GJ, args);
        default: return cudaErrorInvalidValue;
    }
}

struct StepLaunch {
    const DenseArgs *a;
    int W;
    cudaStream_t st;
    bool prepare_only;
};
template <int R, int GJ>
struct StepOp {
    using Args = StepLaunch;
    static cudaError_t run(StepLaunch &L) {
        if (L.W % GJ != 0 || L.W * 32 > DenseBounds<R>::threads) return cudaErrorInvalidValue;
        const int rows_cta = (L.W / GJ) * R;
        const size_t smem = dense_step_smem_bytes(L.a->c.n_pad, R, L.W, GJ);
        if (L.prepare_only)
            return cudaFuncSetAttribute(dense_step_kernel<R, GJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const int grid = (L.a->c.n + rows_cta - 1) / rows_cta;
        return launch_k(dense_step_kernel<R, GJ>, dim3(grid), dim3(L.W * 32), smem, L.st, L.a->c.pdl != 0, *L.a);
    }
};

struct PersistLaunch {
    const PersistArgs *a;
    int W;
    cudaStream_t st;
    bool launch;
    int *grid_out;
};
template <int R, int GJ>
struct PersistOp {
    using Args = PersistLaunch;
    static cudaError_t run(PersistLaunch &L) {
        if (L.W % GJ != 0 || L.W * 32 > PersistBounds<R>::threads) return cudaErrorInvalidValue;
        const int rows_cta = (L.W / GJ) * R;
        const int grid = (L.a->c.n + rows_cta - 1) / rows_cta;
        // the tiles and partials, then the rows' state copy (15 + 4 words) and currents
        const size_t smem = dense_smem_bytes(L.a->c.n_pad, R, L.W) + (size_t)(NCW + 5) * rows_cta * sizeof(float);
        if (!L.launch) {   // prepare, and report whether every CTA can be resident at once
            cudaError_t e = cudaFuncSetAttribute(dense_persist_kernel<R, GJ>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            int per_sm = 0, dev = 0, sms = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense_persist_kernel<R, GJ>, L.W * 32, smem);
            if (e != cudaSuccess) return e;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            *L.grid_out = (grid <= per_sm * sms) ? grid : -grid;
            return cudaSuccess;
        }
        void *args[] = {const_cast<PersistArgs *>(L.a)};
        return cudaLaunchCooperativeKernel((const void *)dense_persist_kernel<R, GJ>, dim3(grid), dim3(L.W * 32), args,
                                           smem, L.st);
    }
};

cudaError_t launch_dense_step(const DenseArgs &a, int R, int W, int GJ, cudaStream_t st) {
    StepLaunch L{&a, W, st, false};
    return dispatch<StepOp>(R, GJ, L);
}

// Raise the kernel's dynamic shared-memory limit (done once, outside stream capture).
cudaError_t prepare_dense_step(int R, int W, int GJ, int n_pad) {
    DenseArgs a{};
    a.c.n_pad = n_pad;
    StepLaunch L{&a, W, nullptr, true};
    return dispatch<StepOp>(R, GJ, L);
}

// launch == false: prepare and check only; *grid_out = grid if every CTA can be resident,
// else -grid.  launch == true: cooperative launch on `st`.
cudaError_t persist_dense(const PersistArgs &a, int R, int W, int GJ, int *grid_out, bool launch, cudaStream_t st) {
    int dummy = 0;
    PersistLaunch L{&a, W, st, launch, grid_out ? grid_out : &dummy};
    return dispatch<PersistOp>(R, GJ, L);
}

int dense_max_threads(int R) { return R <= 4 ? 1024 : 768; }
int persist_max_threads(int R) { return R <= 4 ? 896 : 576; }

}  // namespace ion
