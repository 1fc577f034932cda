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
// FFMA2).  The warps of the first row group also sum the x_j of the real columns (the
// linear part's sum_j u_j).  Lane sums are folded into Kahan-compensated accumulators
// every 64 columns, then summed pairwise across lanes (a fixed butterfly) and across
// column splits, so results are deterministic.
//
// The fused step then runs the explicit-Euler cell update of the CTA's rows, spread over
// NROLE threads per cell (the dendrite, the soma and axon voltages, and groups of gates:
// see cell_step_role), from the rows' state words that cp.async copied into shared memory
// while the pair loop ran; it writes V_dend(t+1) to the other V_dend buffer.
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
    if (!gj_pass<R, GJ>(sm, vcur, n, c.n_pad, bar, uses, m_shift, ui, csp, lane, a.kahan, rg == 0, tot, Us, Uc)) {
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
    // each cell's outputs spread over NROLE threads (a warp holds one role of 32 rows)
    const int rows32 = (rows_cta + 31) & ~31;
    for (int q = threadIdx.x; q < NROLE * rows32; q += blockDim.x) {
        const int role = q / rows32, rr = q - role * rows32;
        const int i = row_base + rr;
        if (rr >= rows_cta || i >= n) continue;
        float iapp = 0.0f;
        if (role == 0) {
            iapp = pulse_current(c.pulses, i, t);
            if (c.iapp != nullptr) iapp += c.iapp[i];
        }
        cell_step_role(role, c, t, vnext, i, staged_cell(cs, rows_cta, rr), ic_s[rr], iapp);
    }
}

// ---- persistent: many steps in one cooperative launch ------------------------------------
// Each row thread keeps its cell's state in registers across steps.  After the cell
// update the new V_dend goes to the other global V_dend buffer and the CTAs meet at a
// bounded grid barrier before staging it for the next step.  With a single CTA and a
// single tile (small networks) V_dend never leaves shared memory: the row threads
// write V_dend(t+1) straight into the tile.
// Launch bounds of the persistent variant (it also keeps a cell's state in registers):
// 896 threads (72 registers) when R <= 2, else 576.
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
    const int rg = warp % GR, cs = warp / GR;
    const int rows_cta = GR * R;
    const DenseSmem sm = dense_smem(smem_raw, c.n_pad);
    const bool single = gridDim.x == 1 && sm.n_tiles == 1;
    const int row_base = blockIdx.x * rows_cta;
    const int64_t t0 = *c.t_dev;

    // row thread: state of one cell in registers
    const int my_row = row_base + (int)threadIdx.x;
    const bool row_thread = threadIdx.x < rows_cta && my_row < n;
    Cell cell{};
    float o_ms = 0.0f, o_ma = 0.0f, o_icah = 0.0f, o_ic = 0.0f;   // last step's output-only words
    int32_t p0 = 0, p1 = 0;
    if (row_thread) {
        cell = load_cell(c.S, vd_slot(c.S, t0), my_row);
        if (c.pulses.off != nullptr) {
            p0 = c.pulses.off[my_row];
            p1 = c.pulses.off[my_row + 1];
        }
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

    bool ok = true;
    for (int k = 0; k < a.n_steps && ok; ++k) {
        const int64_t t = t0 + k;
        const float *vcur = vd_slot(c.S, t);
        if (!single && threadIdx.x == 0)
            for (int q = 0; q < 2 && q < sm.n_tiles; ++q) issue_tile(sm, vcur, c.n_pad, q, bar);
        // shift m = V_dend of cell 0 at step t (from L2, or from the tile itself)
        if (threadIdx.x == 0) m_sh = single ? sm.tile0[0] : __ldcg(vcur);
        __syncthreads();
        const float m_shift = m_sh;
        float ui[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = row_base + rg * R + r;
            ui[r] = (i < n) ? ((single ? sm.tile0[i] : __ldcg(vcur + i)) - m_shift) * GJ_SCALE : 0.0f;
        }
        float tot[R], Us, Uc;
        if (!gj_pass<R, GJ>(sm, single ? nullptr : vcur, n, c.n_pad, bar, uses, m_shift, ui, cs, lane, a.kahan,
                            rg == 0, tot, Us, Uc)) {
            if (threadIdx.x == 0) {
                atomicOr(c.status, (uint32_t)ST_TIMEOUT);
                atomicExch(a.abort_flag, 1u);
                for (int q = 0; q < 2 && q < sm.n_tiles; ++q) (void)mbar_wait_bounded(&bar[q], uses[q] & 1u);
            }
            ok = false;
            break;
        }
        const float U = gj_reduce<R, GJ>(sm, tot, Us, Uc, rg, cs, lane, red_s, red_c, &U_sh);
        if (row_thread) {
            const float u_i = (cell.vd - m_shift) * GJ_SCALE;
            const float ic = row_current<GJ>(sm, (int)threadIdx.x, u_i, n, U, a.g);
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
        }
        if (single) {
            __syncthreads();                          // all pair loops are done with the tile
            if (row_thread) sm.tile0[my_row] = cell.vd;
            __syncthreads();
        } else {
            if (row_thread) vd_slot(c.S, t + 1)[my_row] = cell.vd;
            ok = grid_barrier(a.bar_count, a.abort_flag, a.bar_base + (uint32_t)(k + 1) * gridDim.x, a.timeout_ns, c.status,
                              &ok_sh);
        }
    }
    // write the final state (after an aborted run: the last completed step)
    if (row_thread && a.n_steps > 0) {
        const CellNext o{cell.vd, cell.vs, cell.va, cell.ca, cell.r, cell.s, cell.q, cell.k, cell.l, o_ms,
                         cell.hs, cell.ns, cell.xs, o_ma, cell.ha, cell.xa, o_icah, o_ic};
        store_cell(c.S, vd_slot(c.S, t0 + a.n_steps), my_row, o);
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
        const size_t smem = dense_smem_bytes(L.a->c.n_pad, R, L.W);
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
