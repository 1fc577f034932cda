// ion_ext.cu -- per-flag extensions of a simulation handle (persistent dense launches,
// surrogate) and the batched / training entry points.
#include <cuda_runtime.h>

#include <algorithm>

#include "ion.h"
#include "ion_sim.h"

using namespace ion;

// ---- persistent dense launches ----------------------------------------------------------
// Arrival counter := barrier_base (0 unless a test moved it near 2^32), abort word := 0.
// The barriers compare the counter with their targets modulo 2^32, so a launch may run
// any number of steps whatever the base.
// Barrier words: [0] arrival counter, [1] abort word, [32] release flag (its own 128-byte
// line).  Counter and flag start at barrier_base, the abort word at 0.
constexpr int BAR_WORDS = 64, BAR_FLAG = 32;
static cudaError_t reset_barrier(ion_sim *s) {
    for (int q = 0; q < BAR_WORDS; ++q) s->bar_init[q] = 0u;
    s->bar_init[0] = s->barrier_base;
    s->bar_init[BAR_FLAG] = s->barrier_base;
    return cudaMemcpyAsync(s->d_bar, s->bar_init, BAR_WORDS * sizeof(uint32_t), cudaMemcpyHostToDevice, s->st);
}

// Multi-CTA networks use the half-work kernel (each unordered pair once, two barriers per
// step); one-CTA networks the full-work kernel with V_dend kept in shared memory.
static ion_status half_run(ion_sim *s, int64_t n_steps, const float *iapp) {
    (void)iapp;
    int64_t done = 0;
    while (done < n_steps) {
        const int chunk = (int)std::min<int64_t>(n_steps - done, 1 << 22);
        HalfArgs a{};
        a.c = ion_step_common(s, 0, nullptr);
        a.c.par = -1;   // many steps per launch: the slots follow the device counter
        a.g = s->g;
        a.n_steps = chunk;
        a.rows = (s->persist_W / s->persist_GJ) * s->persist_R;
        a.bar_count = s->d_bar;
        a.abort_flag = s->d_bar + 1;
        a.timeout_ns = s->barrier_timeout_ns;
        a.debug_delay_ns = s->debug_delay_ns;
        a.bar_base = s->barrier_base;
        a.colsum = s->d_half;
        a.colsum_stride = s->half_stride;
        a.usum = s->d_half + (int64_t)s->half_grid * s->half_stride;
        cudaError_t e = reset_barrier(s);
        if (e == cudaSuccess)
            e = launch_dense_half(a, s->persist_R, s->persist_W, s->persist_GJ, s->half_grid, true, nullptr, s->st);
        s->launches++;
        if (e == cudaSuccess) e = launch_advance(s->d_t, chunk, s->st);
        s->launches++;
        if (e != cudaSuccess) return ion_fail(s, ION_ERR_CUDA, "persistent launch: %s", cudaGetErrorString(e));
        done += chunk;
    }
    return ION_OK;
}

static ion_status persist_run(ion_sim *s, int64_t n_steps, const float *iapp) {
    (void)iapp;
    int64_t done = 0;
    while (done < n_steps) {
        const int chunk = (int)std::min<int64_t>(n_steps - done, 1 << 24);
        PersistArgs a{};
        a.c = ion_step_common(s, 0, nullptr);
        a.c.par = -1;   // many steps per launch: the slots follow the device counter
        a.g = s->g;
        a.n_steps = chunk;
        a.kahan = 1;
        a.bar_count = s->d_bar;
        a.abort_flag = s->d_bar + 1;
        a.bar_flag = s->d_bar + BAR_FLAG;
        a.timeout_ns = s->barrier_timeout_ns;
        a.debug_delay_ns = s->debug_delay_ns;
        a.bar_base = s->barrier_base;
        cudaError_t e = reset_barrier(s);
        if (e == cudaSuccess) e = persist_dense(a, s->persist_R, s->persist_W, s->persist_GJ, nullptr, true, s->st);
        s->launches++;
        if (e == cudaSuccess) e = launch_advance(s->d_t, chunk, s->st);
        s->launches++;
        if (e != cudaSuccess) return ion_fail(s, ION_ERR_CUDA, "persistent launch: %s", cudaGetErrorString(e));
        done += chunk;
    }
    return ION_OK;
}

// Shape of a persistent launch: one CTA of ceil(n / 8) warps (8 rows each, one column
// split) when n <= 144, so small networks keep V_dend in shared memory; else the
// per-step shape, if the persistent kernel allows that many threads and all its CTAs
// can be resident at once.
static bool choose_persist_shape(ion_sim *s) {
    PersistArgs probe{};
    probe.c.n = s->n;
    probe.c.n_pad = s->n_pad;
    int R, W, GJ;
    if (s->n <= 144) {
        R = 8;
        W = (s->n + 7) / 8;
        GJ = 1;
    } else {
        R = s->dense_R;
        W = s->dense_W;
        GJ = s->dense_GJ;
        if (W * 32 > persist_max_threads(R)) return false;
    }
    int grid = 0;
    if (persist_dense(probe, R, W, GJ, &grid, false, s->st) != cudaSuccess || grid <= 0) return false;
    s->persist_R = R;
    s->persist_W = W;
    s->persist_GJ = GJ;
    return true;
}

ion_status ion_sim_setup_extras(ion_sim *s, const ion_params *p) {
    s->debug_delay_ns = p->debug_delay_ns;
    s->barrier_base = p->debug_barrier_base;
    if (s->flags & ION_FLAG_SURROGATE) return ion_setup_surrogate(s, p);
    if ((s->flags & ION_FLAG_PERSISTENT) && s->kind == ION_DENSE_UNIFORM && !(s->flags & ION_FLAG_SPLIT)) {
        int coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device);
        if (coop && choose_persist_shape(s)) {
            if (ion_alloc(&s->d_bar, BAR_WORDS * sizeof(uint32_t)) != cudaSuccess)
                return ion_fail(nullptr, ION_ERR_OOM, "persistent: barrier allocation failed");
            s->extra_free = [](ion_sim *q) {   // set before any later allocation can fail
                cudaFree(q->d_bar);
                cudaFree(q->d_half);
                q->d_bar = nullptr;
                q->d_half = nullptr;
            };
            s->run_override = persist_run;
            // several CTAs: the half-work kernel, if its shape and grid fit
            const int rows = (s->persist_W / s->persist_GJ) * s->persist_R;
            const int grid = (s->n + rows - 1) / rows;
            if (grid >= 2 && s->persist_R <= 4 && s->persist_W <= 28 && (s->flags & ION_FLAG_HALF_WORK)) {
                HalfArgs probe{};
                probe.rows = rows;
                int fits = 0;
                if (launch_dense_half(probe, s->persist_R, s->persist_W, s->persist_GJ, grid, false, &fits, s->st) ==
                        cudaSuccess &&
                    fits) {
                    s->half_grid = grid;
                    s->half_stride = half_colsum_stride(grid, rows);
                    if (ion_alloc(&s->d_half, ((size_t)grid * s->half_stride + grid) * sizeof(float)) != cudaSuccess)
                        return ion_fail(nullptr, ION_ERR_OOM, "persistent: column-sum buffer allocation failed");
                    s->run_override = half_run;
                }
            }
        }
    }
    return ION_OK;
}

