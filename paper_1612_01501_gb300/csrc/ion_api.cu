// ion_api.cu -- host side of the C ABI declared in include/ion.h.
//
// A handle owns: the structure-of-arrays state (19 fields plus a second V_dend slot,
// every field padded to a multiple of 256 floats), the connectivity (copied from the
// host or borrowed from the device), a device step counter, a sticky status word, the
// evoked-input table and an optional V_axon trace ring.  Steps are enqueued on the
// caller's stream; chunks of `graph_steps` steps are captured once into a CUDA graph
// and replayed (Sec. 2.4.3 of the paper: the device needs no host data while it runs).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "ion.h"
#include "ion_kernels.cuh"
#include "ion_sim.h"

using namespace ion;

namespace {
thread_local std::string g_last_error;

// The library's constants table (its own copy; the oracle keeps another).  Order of
// enum ion_param.  Entries 0..19 are the 20 conductances of Table "reqs".
const double kModelDefault[ION_NPARAMS] = {
    0.13, 0.25, 0.15,            // g_int, p1 (soma share), p2 (axon share)
    4.5, 35.0, 0.125, 0.016,     // g_CaH, g_KCa, g_h, g_ld
    0.68, 150.0, 9.0, 5.0, 0.016,// g_CaL, g_Na_s, g_Kdr_s, g_K_s, g_ls
    240.0, 20.0, 0.016,          // g_Na_a, g_K_a, g_la
    55.0, -75.0, 120.0, -43.0, 10.0,  // V_Na, V_K, V_Ca, V_h, V_L
    1.0,                         // C_m
    3.0, 0.075,                  // [Ca] influx per unit I_CaH, [Ca] decay rate
    -60.0, 3.715                 // default V_0, [Ca]_0
};
}  // namespace

// ---- errors -------------------------------------------------------------------------
ion_status ion_fail(ion_sim *s, ion_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    g_last_error = buf;
    return code;
}

#define ION_CK(sim, call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return ion_fail((sim), e_ == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA,   \
                            "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

ModelF ion_model_to_f32(const ion_model &m, double dt) {
    const double *v = m.v;
    ModelF P;
    P.g_ds = (float)(v[ION_P_GINT] / (1.0 - v[ION_P_P1]));
    P.g_sd = (float)(v[ION_P_GINT] / v[ION_P_P1]);
    P.g_sa = (float)(v[ION_P_GINT] / (1.0 - v[ION_P_P2]));
    P.g_as = (float)(v[ION_P_GINT] / v[ION_P_P2]);
    P.gCaH = (float)v[ION_P_GCAH];
    P.gKCa = (float)v[ION_P_GKCA];
    P.gh = (float)v[ION_P_GH];
    P.gld = (float)v[ION_P_GLD];
    P.gNas = (float)v[ION_P_GNAS];
    P.gKdrs = (float)v[ION_P_GKDRS];
    P.gKs = (float)v[ION_P_GKS];
    P.gls = (float)v[ION_P_GLS];
    P.gNaa = (float)v[ION_P_GNAA];
    P.gKa = (float)v[ION_P_GKA];
    P.gla = (float)v[ION_P_GLA];
    P.VNa = (float)v[ION_P_VNA];
    P.VK = (float)v[ION_P_VK];
    P.VCa = (float)v[ION_P_VCA];
    P.Vh = (float)v[ION_P_VH];
    P.VL = (float)v[ION_P_VL];
    P.dt_cm = (float)(dt / v[ION_P_CM]);
    P.dt = (float)dt;
    P.ca_in = (float)v[ION_P_CA_IN];
    P.ca_out = (float)v[ION_P_CA_OUT];
    return P;
}

// Per-cell constants (host, ION_NCELLPARAMS x n in ion_param order) to the kernels' per-cell
// rows (ModelF members 0..19, FP32, derived coupling conductances computed in double).
// The g_CaL row is not read.  Rejects non-finite values and area ratios outside (0, 1).
ion_status ion_cell_params_to_f32(const float *cp, int32_t n, const ion_model &m, double dt, std::vector<float> &out) {
    out.assign((size_t)NCELLP * n, 0.0f);
    for (int32_t i = 0; i < n; ++i) {
        ion_model q = m;
        for (int p = 0; p < ION_NCELLPARAMS; ++p) {
            if (p == ION_P_GCAL) continue;
            const float v = cp[(size_t)p * n + i];
            if (!std::isfinite(v))
                return ion_fail(nullptr, ION_ERR_INVALID_ARG, "per-cell constant %d of cell %d not finite", p, i);
            q.v[p] = v;
        }
        if (!(q.v[ION_P_P1] > 0 && q.v[ION_P_P1] < 1 && q.v[ION_P_P2] > 0 && q.v[ION_P_P2] < 1))
            return ion_fail(nullptr, ION_ERR_INVALID_ARG, "per-cell area ratios of cell %d outside (0, 1)", i);
        const ModelF P = ion_model_to_f32(q, dt);
        const float row[NCELLP] = {P.g_ds, P.g_sd, P.g_sa, P.g_as, P.gCaH, P.gKCa, P.gh, P.gld, P.gNas, P.gKdrs,
                                   P.gKs, P.gls, P.gNaa, P.gKa, P.gla, P.VNa, P.VK, P.VCa, P.Vh, P.VL};
        for (int k = 0; k < NCELLP; ++k) out[(size_t)k * n + i] = row[k];
    }
    return ION_OK;
}

static bool model_valid(const ion_model &m) {
    for (double x : m.v)
        if (!std::isfinite(x)) return false;
    return m.v[ION_P_P1] > 0 && m.v[ION_P_P1] < 1 && m.v[ION_P_P2] > 0 && m.v[ION_P_P2] < 1 && m.v[ION_P_CM] > 0;
}

extern "C" void ion_model_default(ion_model *out) {
    if (out) std::memcpy(out->v, kModelDefault, sizeof kModelDefault);
}

extern "C" const char *ion_last_error(const ion_sim *s) {
    return s ? s->err.c_str() : g_last_error.c_str();
}

static bool csr_use16(const ion_sim *s, bool staged);

extern "C" ion_status ion_csr_layout(const ion_sim *s, int32_t *index_bytes, int32_t *weight_bytes, int32_t *staged) {
    if (!s) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_csr_layout: NULL handle");
    const bool csr = s->kind == ION_CSR && !s->d_map;
    const bool c16 = csr && csr_use16(s, s->csr_staged != 0);
    if (index_bytes) *index_bytes = csr ? (c16 ? 2 : 4) : 0;
    if (weight_bytes) *weight_bytes = csr && s->d_w ? 4 : 0;
    if (staged) *staged = csr ? s->csr_staged : 0;
    return ION_OK;
}

extern "C" int64_t ion_step_count(const ion_sim *s) { return s ? s->t : -1; }
extern "C" int64_t ion_launch_count(const ion_sim *s) { return s ? s->launches : -1; }

// ---- model probes -------------------------------------------------------------------
extern "C" ion_status ion_rates(float V, float ca, float *xinf, float *tau) {
    if (!xinf || !tau) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_rates: NULL output");
    float *d = nullptr;
    ION_CK(nullptr, ion_alloc(&d, 2 * NG * sizeof(float)));
    cudaError_t e = launch_rates(V, ca, d, 0);
    float h[2 * NG];
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "ion_rates: %s", cudaGetErrorString(e));
    std::memcpy(xinf, h, NG * sizeof(float));
    std::memcpy(tau, h + NG, NG * sizeof(float));
    return ION_OK;
}

extern "C" ion_status ion_default_state(const ion_model *model, int32_t n, float *out) {
    if (!out || n < 1) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_default_state: bad arguments");
    ion_model m;
    if (model) m = *model;
    else ion_model_default(&m);
    if (!model_valid(m)) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_default_state: invalid model table");
    float *d = nullptr;
    ION_CK(nullptr, ion_alloc(&d, (size_t)NF * n * sizeof(float)));
    const ModelF P = ion_model_to_f32(m, 0.05);
    cudaError_t e = launch_default_state(P, (float)m.v[ION_P_V0], (float)m.v[ION_P_CA0], (float)m.v[ION_P_GCAL], n, n,
                                         d, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, (size_t)NF * n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "ion_default_state: %s", cudaGetErrorString(e));
    return ION_OK;
}

// ---- device allocation (with the test hook) ------------------------------------------
static std::atomic<int64_t> g_fail_after{-1};   // allocations left before the injected failure

cudaError_t ion_dev_alloc(void **p, size_t bytes) {
    int64_t k = g_fail_after.load();
    while (k >= 0) {
        if (g_fail_after.compare_exchange_weak(k, k - 1)) {
            if (k == 0) {   // this call fails, once
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

extern "C" ion_status ion_debug_fail_alloc(int32_t after) {
    g_fail_after.store(after < 0 ? -1 : (int64_t)after);
    return ION_OK;
}

// ---- validation --------------------------------------------------------------------
ion_status ion_validate_csr(int32_t n, const ion_conn *c) {
    const int32_t *rp = c->row_ptr, *col = c->col_idx;
    if (!rp || (c->nnz > 0 && !col)) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "CSR: NULL row_ptr/col_idx");
    if (c->nnz < 0 || c->nnz >= (int64_t)INT32_MAX) return ion_fail(nullptr, ION_ERR_BAD_CSR, "CSR: nnz out of range");
    if (c->mem == ION_DEVICE) return ION_OK;  // device arrays are trusted (documented)
    if (rp[0] != 0) return ion_fail(nullptr, ION_ERR_BAD_CSR, "CSR: row_ptr[0] = %d, expected 0", rp[0]);
    if ((int64_t)rp[n] != c->nnz)
        return ion_fail(nullptr, ION_ERR_BAD_CSR, "CSR: row_ptr[n] = %d but nnz = %lld", rp[n], (long long)c->nnz);
    for (int32_t i = 0; i < n; ++i) {
        if (rp[i + 1] < rp[i]) return ion_fail(nullptr, ION_ERR_BAD_CSR, "CSR: row_ptr decreases at row %d", i);
        if ((int64_t)rp[i + 1] > c->nnz) return ion_fail(nullptr, ION_ERR_BAD_CSR, "CSR: row_ptr[%d] beyond nnz", i + 1);
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t j = col[e];
            if (j < 0 || j >= n) return ion_fail(nullptr, ION_ERR_BAD_CSR, "CSR: col_idx[%d] = %d out of range", e, j);
            if (j == i) return ion_fail(nullptr, ION_ERR_BAD_CSR, "CSR: self loop at row %d", i);
            if (e > rp[i] && col[e - 1] >= j)
                return ion_fail(nullptr, ION_ERR_BAD_CSR, "CSR: row %d not strictly ascending", i);
        }
    }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t j = col[e];
            if (!std::binary_search(col + rp[j], col + rp[j + 1], i))
                return ion_fail(nullptr, ION_ERR_BAD_CSR, "CSR: not symmetric (%d -> %d has no reverse)", i, j);
        }
    if (c->weight)
        for (int64_t e = 0; e < c->nnz; ++e)
            if (!std::isfinite(c->weight[e])) return ion_fail(nullptr, ION_ERR_BAD_CSR, "CSR: weight %lld not finite", (long long)e);
    return ION_OK;
}

// ---- launch-shape choice -----------------------------------------------------------
static int num_sms() {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Dense: a CTA has W = GR x GJ warps (GR row groups of R rows, GJ column splits) and
// owns GR * R rows.  Pick (R, GR, GJ) to minimise the work of the busiest SM,
// ceil(grid / SMs) * (GR * R + 4): every row costs the same N pair evaluations and every
// CTA pays about four rows' worth for staging and scaling its V_dend tiles.  Among equal
// costs prefer 24..32 warps per CTA (the SFU pipe needs that many warps in flight; a
// probe of the pair loop gave 0.44 / 0.67 / 0.77 of the ex2 peak at 9 / 18 / 32 warps),
// then fewer rows per warp (a smaller register footprint).
void ion_choose_dense_shape(int n, int sms, int *R_out, int *W_out, int *GJ_out) {
    static const int Rs[] = {1, 2, 4, 6, 8};
    static const int GJs[] = {1, 2, 4};
    long best_cost = -1;
    int best_score = -1;
    int bR = 1, bW = 1, bGJ = 1;
    for (int R : Rs)
        for (int GJ : GJs)
            for (int GR = 1; GR <= 32; ++GR) {
                const int W = GR * GJ;
                if (W * 32 > dense_max_threads(R)) continue;
                const long rows = (long)GR * R;
                const long grid = (n + rows - 1) / rows;
                const long cost = ((grid + sms - 1) / sms) * (rows + 4);
                const int warps_score = (W >= 24) ? 3 : (W >= 16 ? 2 : (W >= 8 ? 1 : 0));
                const int score = warps_score * 16 + (8 - R);
                if (best_cost < 0 || cost < best_cost || (cost == best_cost && score > best_score)) {
                    best_cost = cost;
                    best_score = score;
                    bR = R;
                    bW = W;
                    bGJ = GJ;
                }
            }
    *R_out = bR;
    *W_out = bW;
    *GJ_out = bGJ;
}

// CSR: lanes per row from the mean degree (about two edges per lane per pass, four per
// lane for the densest rows), and rows per CTA so that a row group's work per CTA stays
// near 2-8 K edges and the grid has several CTAs per SM.
void ion_choose_csr_shape(double mean_deg, int *SW, int *rows) {
    int sw = 32;
    if (mean_deg <= 3) sw = 1;
    else if (mean_deg <= 6) sw = 2;
    else if (mean_deg <= 12) sw = 4;
    else if (mean_deg <= 40) sw = 8;
    else if (mean_deg <= 120) sw = 16;
    *SW = sw;
    int r = 256;
    if (mean_deg > 48) r = 128;
    if (mean_deg > 192) r = 64;
    if (mean_deg > 384) r = 32;
    *rows = r;
}

// Shared-memory staging of V_dend for a CSR network (mode 0: choose, 1: off, 2: on).
// Staging pays when rows are long: a warp's 32 random gathers then cost about 3.8
// shared-memory wavefronts instead of 32 L1 lines.  Measured: the 65 536-cell network at
// k = 1000 went from 0.45 to 0.69 of HBM bandwidth (32-bit columns), k = 100 from 20.6 to
// 16.9 us per step (16-bit columns), and random networks of 10 000-13 000 cells at 25-50 %
// density ran about twice as fast staged.  The default stages rows of 64 or more edges that
// keep 32 or more per chunk, or any CSR too large for L2 (over 96 MB) with rows of 64 or
// more edges; rows of ~10 edges stay on the direct kernel.  One CTA per SM owns ceil(n / SMs) rows (at most
// 1024).  Only
// CSR arrays copied from the host are staged: their columns were checked to be sorted
// and in range, which the chunk boundaries rely on.
// The 16-bit columns serve the staged kernel (columns relative to a chunk of at most 2^16
// cells) and the direct kernel when n <= 65 536 and rows are long enough (mean degree >= 32)
// for its eight-edge groups; shorter rows read 32-bit columns four at a time.
static bool csr_use16(const ion_sim *s, bool staged) {
    if (s->d_col16 == nullptr || s->d_rev != nullptr) return false;   // the half-work passes read 32-bit columns
    return staged || (s->n <= 65536 && s->nnz >= 32 * (int64_t)s->n);
}

// Connectivity fields of a CSR launch.
void ion_csr_fill(const ion_sim *s, CsrArgs &a, bool staged) {
    a.row_ptr = s->d_rowptr;
    a.col = s->d_col;
    a.w = s->d_w;
    a.g = s->g;
    a.col16 = csr_use16(s, staged) ? s->d_col16 : nullptr;
    if (staged && s->d_col16p && a.col16 && s->pad_rows == s->csr_chunk_rows) {
        a.col16p = s->d_col16p;
        a.wp = s->d_wp;
        a.segoff = s->d_segoff;
    }
}

// The staged kernel's padded layout (see ion_sim): segment offsets on the host from the row
// pointers and chunk boundaries, the columns and weights by a fill kernel.
static ion_status build_padded_layout(ion_sim *s) {
    const int n = s->n, C = s->n_chunks, rows = s->csr_chunk_rows;
    std::vector<int32_t> rp((size_t)n + 1), mid((size_t)(C - 1) * n);
    cudaError_t e = cudaMemcpyAsync(rp.data(), s->d_rowptr, rp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess && C > 1)
        e = cudaMemcpyAsync(mid.data(), s->d_mid, mid.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "CSR padded layout: %s", cudaGetErrorString(e));
    std::vector<int32_t> off((size_t)C * n + 1);
    int64_t tot = 0;
    for (int ch = 0; ch < C; ++ch)
        for (int i = 0; i < n; ++i) {
            const int64_t b = ch == 0 ? rp[i] : mid[(size_t)(ch - 1) * n + i];
            const int64_t en = ch == C - 1 ? rp[i + 1] : mid[(size_t)ch * n + i];
            off[(size_t)ch * n + i] = (int32_t)tot;
            tot += (en - b + 7) & ~(int64_t)7;
            if (tot >= INT32_MAX) return ION_OK;   // too large for 32-bit offsets: keep the unpadded layout
        }
    off[(size_t)C * n] = (int32_t)tot;
    e = ion_alloc(&s->d_segoff, off.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = ion_alloc(&s->d_col16p, (size_t)std::max<int64_t>(tot, 8) * sizeof(uint16_t));
    if (e == cudaSuccess && s->d_w) e = ion_alloc(&s->d_wp, (size_t)std::max<int64_t>(tot, 8) * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_segoff, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess)
        e = launch_csr_pad_fill(s->d_rowptr, s->d_mid, s->d_col, s->d_w, n, C, rows, std::min(CSR_CHUNK, s->n_pad),
                                s->d_segoff, s->d_col16p, s->d_wp, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);   // the host offsets are released on return
    if (e != cudaSuccess) {
        cudaFree(s->d_segoff);
        cudaFree(s->d_col16p);
        cudaFree(s->d_wp);
        s->d_segoff = nullptr;
        s->d_col16p = nullptr;
        s->d_wp = nullptr;
        return ion_fail(nullptr, e == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA, "CSR padded layout: %s",
                        cudaGetErrorString(e));
    }
    s->pad_rows = rows;
    return ION_OK;
}

ion_status ion_setup_csr_staging(ion_sim *s, int mode) {
    const double deg = s->n > 0 ? (double)s->nnz / s->n : 0.0;
    const double csr_bytes = (double)((s->d_col16 ? 2 : 4) + (s->d_w ? 4 : 0)) * (double)s->nnz;
    const double chunks = (double)((s->n_pad + CSR_CHUNK - 1) / CSR_CHUNK);
    const bool on = mode == 2 || (mode == 0 && deg >= 64.0 && (csr_bytes > 96.0e6 || deg / chunks >= 32.0));
    s->csr_staged = 0;
    // staging relies on validated (sorted, in-range) columns: host-copied CSR only
    // (the surrogate path computes its gap currents with the direct kernel)
    if (!on || (s->flags & (ION_FLAG_SPLIT | ION_FLAG_SURROGATE)) || !s->own_csr || s->d_rev) return ION_OK;
    s->n_chunks = (s->n_pad + CSR_CHUNK - 1) / CSR_CHUNK;
    int rows = (s->n + s->sms - 1) / s->sms;
    if (rows > 1024) rows = 1024;
    if (rows < 1) rows = 1;
    int sw, r_unused;
    ion_choose_csr_shape(deg / s->n_chunks, &sw, &r_unused);
    if (s->csr_chunk_rows == 0) s->csr_chunk_rows = rows;
    s->csr_chunk_SW = sw;
    if (s->n_chunks > 1 && !s->d_mid) {
        cudaError_t e = ion_alloc(&s->d_mid, (size_t)(s->n_chunks - 1) * s->n * sizeof(int32_t));
        if (e == cudaSuccess) e = launch_csr_chunk_bounds(s->d_rowptr, s->d_col, s->n, s->n_chunks, s->d_mid, s->st);
        if (e != cudaSuccess)
            return ion_fail(nullptr, e == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA, "CSR staging setup: %s",
                            cudaGetErrorString(e));
    }
    // The padded layout removes each segment's head and tail (up to 14 edges handled one by
    // one); measured, it pays for segments of up to ~1000 edges with the exponential
    // junction and at every length with the linear one, while exponential-junction rows of
    // several thousand edges per chunk ran 4-9 % slower on it: those keep the unpadded layout.
    const bool pad = (s->flags & ION_FLAG_SGJ) || deg / s->n_chunks <= 1024.0;
    if (pad && s->d_col16 && !s->col16_bank && !s->d_col16p) {
        const ion_status sp = build_padded_layout(s);
        if (sp != ION_OK) return sp;
    }
    const ion_status st = ion_prepare_csr_chunk(s);
    if (st != ION_OK) return st;
    s->csr_staged = 1;
    return ION_OK;
}

// Allow the staged kernel of the current lanes-per-row choice its dynamic shared memory.
ion_status ion_prepare_csr_chunk(ion_sim *s) {
    CsrArgs probe{};
    probe.c.n = s->n;
    probe.c.n_pad = s->n_pad;
    ion_csr_fill(s, probe, true);
    cudaError_t e = launch_csr_chunk_step(probe, s->csr_chunk_SW, s->csr_chunk_rows, s->d_mid, s->n_chunks, true, s->st);
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "CSR staging setup: %s", cudaGetErrorString(e));
    return ION_OK;
}

// ---- creation -------------------------------------------------------------------------
static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Half-work CSR: per row the first upper edge, per upper edge the position of its mirror
// (host binary search in the sorted rows), the slot and upper-sum buffers.  Needs a host
// CSR with symmetric weights (checked bit for bit).
ion_status ion_setup_csr_half(ion_sim *s, const ion_conn *conn) {
    if (conn->mem != ION_HOST)
        return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "half-work CSR needs host arrays");
    if (s->flags & (ION_FLAG_SPLIT | ION_FLAG_SGJ | ION_FLAG_PERSISTENT | ION_FLAG_SURROGATE))
        return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "half-work CSR: not with SPLIT, SGJ, PERSISTENT or SURROGATE");
    const int32_t n = s->n, *rp = conn->row_ptr, *col = conn->col_idx;
    std::vector<int32_t> split((size_t)n), rev((size_t)std::max<int64_t>(s->nnz, 1), 0);
    for (int32_t i = 0; i < n; ++i) {
        split[(size_t)i] = (int32_t)(std::upper_bound(col + rp[i], col + rp[i + 1], i) - col);
        for (int32_t e = split[(size_t)i]; e < rp[i + 1]; ++e) {
            const int32_t j = col[e];
            const int32_t m = (int32_t)(std::lower_bound(col + rp[j], col + rp[j + 1], i) - col);   // (j, i)
            if (conn->weight) {
                uint32_t a, b;
                std::memcpy(&a, conn->weight + e, 4);
                std::memcpy(&b, conn->weight + m, 4);
                if (a != b) return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "half-work CSR needs symmetric weights");
            }
            rev[(size_t)e] = m;
        }
    }
    cudaError_t e = ion_alloc(&s->d_split, (size_t)n * sizeof(int32_t));
    if (e == cudaSuccess) e = ion_alloc(&s->d_rev, rev.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = ion_alloc(&s->d_slot, rev.size() * sizeof(float));
    if (e == cudaSuccess) e = ion_alloc(&s->d_icu, (size_t)s->n_pad * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_split, split.data(), split.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_rev, rev.data(), rev.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);   // the host vectors go out of scope
    if (e != cudaSuccess)
        return ion_fail(nullptr, e == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA, "half-work CSR setup: %s",
                        cudaGetErrorString(e));
    s->lps = 2;
    return ION_OK;
}

void ion_sim_free_device(ion_sim *s) {
    ion_drop_graphs(s);
    cudaFree(s->d_state);
    cudaFree(s->d_t);
    cudaFree(s->d_status);
    if (s->own_csr) {
        cudaFree(s->d_rowptr);
        cudaFree(s->d_col);
        cudaFree(s->d_w);
    }
    cudaFree(s->d_col16);
    s->d_col16 = nullptr;
    cudaFree(s->d_sgj);
    s->d_sgj = nullptr;
    cudaFree(s->d_W);
    s->d_W = nullptr;

    cudaFree(s->d_poff);
    cudaFree(s->d_pbeg);
    cudaFree(s->d_pend);
    cudaFree(s->d_pamp);
    cudaFree(s->d_iapp);
    cudaFree(s->d_trace);
    cudaFree(s->d_ic);
    cudaFree(s->d_cellp);
    s->d_cellp = nullptr;
    cudaFree(s->d_split);
    cudaFree(s->d_rev);
    cudaFree(s->d_slot);
    cudaFree(s->d_icu);
    s->d_split = s->d_rev = nullptr;
    s->d_slot = s->d_icu = nullptr;
    cudaFree(s->d_mid);
    cudaFree(s->d_col16p);
    cudaFree(s->d_wp);
    cudaFree(s->d_segoff);
    cudaFree(s->d_mlp);
    cudaFree(s->d_mlp_tc);
    s->d_mlp_tc = nullptr;
    s->extra_free(s);
}

extern "C" ion_status ion_create(const ion_net *net, const ion_conn *conn, const ion_params *params,
                                 const float *init_state, ion_sim **out) {
    if (!out) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: NULL out");
    *out = nullptr;
    if (!net || !params) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: NULL net/params");
    if (net->n_cells < 1 || net->n_cells > (1 << 28))
        return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: n_cells = %d out of range", net->n_cells);
    if (net->kind != ION_DENSE_UNIFORM && net->kind != ION_CSR && net->kind != ION_NO_GJ &&
        net->kind != ION_DENSE_MATRIX)
        return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: unknown network kind %d", net->kind);
    if (net->kind != ION_NO_GJ && !conn) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: NULL conn");
    if (conn && conn->mem != ION_HOST && conn->mem != ION_DEVICE)
        return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: bad conn.mem");
    if (net->kind == ION_DENSE_UNIFORM && !std::isfinite(conn->g_c))
        return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: g_c not finite");
    if (net->kind == ION_CSR) {
        ion_status st = ion_validate_csr(net->n_cells, conn);
        if (st != ION_OK) return st;
    }
    if (net->kind == ION_DENSE_MATRIX) {
        if (!conn->weight) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: dense matrix without weights");
        if (params->flags & (ION_FLAG_PERSISTENT | ION_FLAG_SURROGATE | ION_FLAG_SPLIT | ION_FLAG_SGJ))
            return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "ion_create: flags not supported with a dense matrix");
        if (conn->mem == ION_HOST)
            for (int64_t q = 0; q < (int64_t)net->n_cells * net->n_cells; ++q)
                if (!std::isfinite(conn->weight[q]))
                    return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: matrix weight %lld not finite", (long long)q);
    }
    if ((params->flags & ION_FLAG_SGJ) &&
        (net->kind == ION_NO_GJ || (params->flags & (ION_FLAG_PERSISTENT | ION_FLAG_SURROGATE | ION_FLAG_SPLIT))))
        return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "ion_create: ION_FLAG_SGJ needs a dense or CSR network "
                        "without PERSISTENT, SURROGATE or SPLIT");
    const double dt = params->dt_ms > 0 ? params->dt_ms : 0.05;
    if (!std::isfinite(dt) || dt > 1.0) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: dt_ms out of range");
    ion_model m;
    if (params->model) m = *params->model;
    else ion_model_default(&m);
    if (!model_valid(m)) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: invalid model table");
    if (params->flags & ION_FLAG_SURROGATE) {
        if (!params->surrogate) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: SURROGATE flag without weights");
    }
    std::vector<float> cellp;   // per-cell constants in the kernels' order (ModelF members 0..19)
    if (params->cell_params) {
        if (net->kind == ION_DENSE_MATRIX ||
            (params->flags & (ION_FLAG_PERSISTENT | ION_FLAG_SURROGATE | ION_FLAG_SGJ)))
            return ion_fail(nullptr, ION_ERR_UNSUPPORTED, "ion_create: per-cell constants need a dense uniform, CSR "
                            "or NO_GJ network without PERSISTENT, SURROGATE or SGJ");
        const ion_status cst = ion_cell_params_to_f32(params->cell_params, net->n_cells, m, dt, cellp);
        if (cst != ION_OK) return cst;
    }

    ion_sim *s = new (std::nothrow) ion_sim();
    if (!s) return ion_fail(nullptr, ION_ERR_OOM, "ion_create: host allocation failed");
    s->n = net->n_cells;
    s->n_user = net->n_cells;
    s->kind = net->kind;
    s->n_pad = (int32_t)round_up(s->n, PAD_J);
    s->stride = s->n_pad;
    s->flags = params->flags;
    s->graph_steps = params->graph_steps > 0 ? params->graph_steps : 50;
    s->check_every = params->check_every > 0 ? params->check_every : 64;
    s->barrier_timeout_ns = params->barrier_timeout_ns ? params->barrier_timeout_ns : 2000000000ull;
    s->st = (cudaStream_t)params->cuda_stream;
    if (s->st == nullptr) {   // no stream given: a private one (graph capture needs a non-legacy stream)
        if (cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return ion_fail(nullptr, ION_ERR_CUDA, "ion_create: could not create a stream");
        }
        s->st = s->own_stream;
    }
    s->model = m;
    s->dt = dt;
    s->P = ion_model_to_f32(m, dt);
    cudaGetDevice(&s->device);
    const int sms = num_sms();
    s->sms = sms;

    auto fail = [&](ion_status code) {
        cudaStreamSynchronize(s->st);   // initialisation kernels already queued finish first
        ion_sim_free_device(s);
        if (s->own_stream) cudaStreamDestroy(s->own_stream);
        delete s;
        return code;
    };
    // state: 20 slots of stride floats (fields 0..18 + second V_dend slot)
    cudaError_t e = ion_alloc(&s->d_state, (size_t)20 * s->stride * sizeof(float));
    if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_OOM, "ion_create: state allocation: %s", cudaGetErrorString(e)));
    e = ion_alloc(&s->d_t, sizeof(int64_t));
    if (e == cudaSuccess) e = ion_alloc(&s->d_status, sizeof(uint32_t));
    if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_OOM, "ion_create: %s", cudaGetErrorString(e)));
    e = cudaMemsetAsync(s->d_state, 0, (size_t)20 * s->stride * sizeof(float), s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_t, 0, sizeof(int64_t), s->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_status, 0, sizeof(uint32_t), s->st);
    // sentinel padding of both V_dend slots (padded pairs contribute exactly zero)
    if (e == cudaSuccess) e = launch_fill(s->d_state + s->n, PAD_VOLT, s->n_pad - s->n, s->st);
    if (e == cudaSuccess) e = launch_fill(s->d_state + 19 * s->stride + s->n, PAD_VOLT, s->n_pad - s->n, s->st);
    if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_CUDA, "ion_create: init: %s", cudaGetErrorString(e)));
    if (init_state) {
        e = cudaMemcpy2DAsync(s->d_state, s->stride * sizeof(float), init_state, s->n * sizeof(float),
                              s->n * sizeof(float), NF, cudaMemcpyHostToDevice, s->st);
    } else {
        e = launch_default_state(s->P, (float)m.v[ION_P_V0], (float)m.v[ION_P_CA0], (float)m.v[ION_P_GCAL], s->n,
                                 s->stride, s->d_state, s->st);
    }
    if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_CUDA, "ion_create: initial state: %s", cudaGetErrorString(e)));

    // connectivity
    if (s->kind == ION_DENSE_UNIFORM) {
        s->g = conn->g_c;
        int R, W, GJ;
        ion_choose_dense_shape(s->n, sms, &R, &W, &GJ);
        const ion_tune *tu = (const ion_tune *)params->tune;
        if (tu && tu->dense_rows_per_warp > 0) R = tu->dense_rows_per_warp;
        if (tu && tu->dense_warps > 0) W = tu->dense_warps;
        if (tu && tu->dense_col_splits > 0) GJ = tu->dense_col_splits;
        if (R != 1 && R != 2 && R != 4 && R != 6 && R != 8)
            return fail(ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: dense_rows_per_warp %d unsupported", R));
        if ((GJ != 1 && GJ != 2 && GJ != 4) || W < 1 || W % GJ != 0 || W * 32 > dense_max_threads(R))
            return fail(ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: dense shape R=%d W=%d GJ=%d unsupported", R, W, GJ));
        s->dense_R = R;
        s->dense_W = W;
        s->dense_GJ = GJ;
        e = prepare_dense_step(R, W, GJ, s->n_pad);
        if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_CUDA, "ion_create: dense setup: %s", cudaGetErrorString(e)));
    } else if (s->kind == ION_DENSE_MATRIX) {
        e = ion_alloc(&s->d_W, (size_t)s->n * s->n_pad * sizeof(float));
        if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_OOM, "ion_create: matrix allocation: %s", cudaGetErrorString(e)));
        e = cudaMemsetAsync(s->d_W, 0, (size_t)s->n * s->n_pad * sizeof(float), s->st);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(s->d_W, (size_t)s->n_pad * sizeof(float), conn->weight, (size_t)s->n * sizeof(float),
                                  (size_t)s->n * sizeof(float), (size_t)s->n,
                                  conn->mem == ION_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st);
        if (e == cudaSuccess) e = prepare_matrix_step(s->n_pad);
        if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_CUDA, "ion_create: matrix copy: %s", cudaGetErrorString(e)));
        s->dense_R = matrix_default_R(s->n, sms);
        const ion_tune *tu = (const ion_tune *)params->tune;
        if (tu && tu->dense_rows_per_warp > 0) s->dense_R = tu->dense_rows_per_warp;
        if (s->dense_R != 1 && s->dense_R != 2 && s->dense_R != 4)
            return fail(ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: matrix rows per warp %d unsupported", s->dense_R));
    } else if (s->kind == ION_CSR) {
        s->g = conn->g_c;
        s->nnz = conn->nnz;
        if (conn->mem == ION_DEVICE) {
            s->own_csr = false;
            s->d_rowptr = const_cast<int32_t *>(conn->row_ptr);
            s->d_col = const_cast<int32_t *>(conn->col_idx);
            s->d_w = const_cast<float *>(conn->weight);
        } else {
            s->own_csr = true;
            const bool compact = !(s->flags & ION_FLAG_CSR_AS_GIVEN);
            // every weight bitwise equal: keep one scalar (the kernels multiply the row sum by it)
            bool keep_w = conn->weight != nullptr && s->nnz > 0;
            if (keep_w && compact) {
                uint32_t b0, be;
                std::memcpy(&b0, conn->weight, sizeof b0);
                bool all = true;
                for (int64_t q = 1; q < s->nnz && all; ++q) {
                    std::memcpy(&be, conn->weight + q, sizeof be);
                    all = be == b0;
                }
                if (all) {
                    s->g = conn->weight[0];
                    keep_w = false;
                }
            }
            e = ion_alloc(&s->d_rowptr, (size_t)(s->n + 1) * sizeof(int32_t));
            if (e == cudaSuccess && s->nnz > 0) e = ion_alloc(&s->d_col, (size_t)s->nnz * sizeof(int32_t));
            if (e == cudaSuccess && keep_w) e = ion_alloc(&s->d_w, (size_t)s->nnz * sizeof(float));
            // the low 16 bits of every column, padded to whole 16-byte groups
            if (e == cudaSuccess && s->nnz > 0 && compact) e = ion_alloc(&s->d_col16, (size_t)round_up(s->nnz, 8) * sizeof(uint16_t));
            if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_OOM, "ion_create: CSR allocation: %s", cudaGetErrorString(e)));
            e = cudaMemcpyAsync(s->d_rowptr, conn->row_ptr, (size_t)(s->n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s->st);
            if (e == cudaSuccess && s->nnz > 0)
                e = cudaMemcpyAsync(s->d_col, conn->col_idx, (size_t)s->nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s->st);
            if (e == cudaSuccess && s->d_w)
                e = cudaMemcpyAsync(s->d_w, conn->weight, (size_t)s->nnz * sizeof(float), cudaMemcpyHostToDevice, s->st);
            if (e == cudaSuccess && s->d_col16) {
                const ion_tune *tb = (const ion_tune *)params->tune;
                std::vector<uint16_t> h16;   // opt-in: bank order (uniform weights only: no weight array to permute)
                if (tb && tb->csr_bank_order == 1 && !keep_w &&
                    ion_csr_bank_col16(s->n, s->n_pad, conn->row_ptr, conn->col_idx, h16)) {
                    e = cudaMemcpy(s->d_col16, h16.data(), h16.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
                    s->col16_bank = true;
                } else
                    e = launch_csr_col16(s->d_col, s->nnz, round_up(s->nnz, 8), s->d_col16, s->st);
            }
            if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_CUDA, "ion_create: CSR copy: %s", cudaGetErrorString(e)));
        }
        if (s->flags & ION_FLAG_HALF_WORK) {
            const ion_status hs = ion_setup_csr_half(s, conn);
            if (hs != ION_OK) return fail(hs);
        }
        int SW, rows;
        ion_choose_csr_shape((double)s->nnz / s->n, &SW, &rows);
        const ion_tune *tu = (const ion_tune *)params->tune;
        if (tu && tu->csr_lanes_per_row > 0) SW = tu->csr_lanes_per_row;
        if (tu && tu->csr_rows_per_cta > 0) rows = tu->csr_rows_per_cta;
        if ((SW & (SW - 1)) != 0 || SW < 1 || SW > 32 || rows < 1 || rows > 256)
            return fail(ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_create: bad CSR launch shape"));
        e = prepare_csr_step();
        if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_CUDA, "ion_create: CSR setup: %s", cudaGetErrorString(e)));
        s->csr_SW = SW;
        s->csr_rows = rows;
        const ion_status st3 = ion_setup_csr_staging(s, tu ? tu->csr_staging : 0);
        if (st3 != ION_OK) return fail(st3);
    }
    if ((s->flags & ION_FLAG_SGJ) && s->kind == ION_DENSE_UNIFORM) {
        s->lps = s->n <= SGJ_ONE_LAUNCH ? 1 : 2;   // (partial sums +) update
        e = ion_alloc(&s->d_sgj, (size_t)sgj_partials(s->n) * sizeof(float));
        if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_OOM, "ion_create: %s", cudaGetErrorString(e)));
    }
    if (!cellp.empty()) {   // per-cell constants: read by the stand-alone cell update
        if (s->kind != ION_NO_GJ) s->flags |= ION_FLAG_SPLIT;
        e = ion_alloc(&s->d_cellp, (size_t)NCELLP * s->stride * sizeof(float));
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(s->d_cellp, s->stride * sizeof(float), cellp.data(), s->n * sizeof(float),
                                  s->n * sizeof(float), NCELLP, cudaMemcpyHostToDevice, s->st);
        if (e != cudaSuccess)
            return fail(ion_fail(nullptr, e == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA,
                                 "ion_create: per-cell constants: %s", cudaGetErrorString(e)));
    }
    if ((s->flags & ION_FLAG_SPLIT) && s->kind != ION_NO_GJ) {
        s->lps = 2;
        e = ion_alloc(&s->d_ic, (size_t)s->n_pad * sizeof(float));
        if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_OOM, "ion_create: %s", cudaGetErrorString(e)));
    }
    ion_status st2 = ion_sim_setup_extras(s, params);
    if (st2 != ION_OK) return fail(st2);
    e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return fail(ion_fail(nullptr, ION_ERR_CUDA, "ion_create: %s", cudaGetErrorString(e)));
    *out = s;
    return ION_OK;
}

extern "C" void ion_destroy(ion_sim *s) {
    if (!s) return;
    cudaStreamSynchronize(s->st);
    if (s->copy_st) {
        cudaStreamSynchronize(s->copy_st);
        cudaStreamDestroy(s->copy_st);
        cudaEventDestroy(s->ev_ready);
        cudaEventDestroy(s->ev_copied);
    }
    ion_sim_free_device(s);
    if (s->own_stream) cudaStreamDestroy(s->own_stream);
    delete s;
}

// ---- evoked input -------------------------------------------------------------------
static ion_status install_pulses(ion_sim *s, const ion_input *in) {
    const int32_t np = in->n_pulses;
    if (np < 0) return ion_fail(s, ION_ERR_INVALID_ARG, "pulses: negative count");
    std::vector<int32_t> cell(np);
    std::vector<int64_t> beg(np), end(np);
    std::vector<float> amp(np);
    if (np > 0) {
        if (!in->pulse_cell || !in->pulse_begin || !in->pulse_end || !in->pulse_amp)
            return ion_fail(s, ION_ERR_INVALID_ARG, "pulses: NULL array");
        const cudaMemcpyKind k = in->mem == ION_DEVICE ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        ION_CK(s, cudaMemcpy(cell.data(), in->pulse_cell, np * sizeof(int32_t), k));
        ION_CK(s, cudaMemcpy(beg.data(), in->pulse_begin, np * sizeof(int64_t), k));
        ION_CK(s, cudaMemcpy(end.data(), in->pulse_end, np * sizeof(int64_t), k));
        ION_CK(s, cudaMemcpy(amp.data(), in->pulse_amp, np * sizeof(float), k));
    }
    for (int32_t p = 0; p < np; ++p) {
        if (cell[p] < 0 || cell[p] >= s->n_user) return ion_fail(s, ION_ERR_INVALID_ARG, "pulse %d: cell %d out of range", p, cell[p]);
        if (s->d_map) cell[p] = ion_batch_map_cell(s, cell[p]);   // user numbering -> padded segments
        if (end[p] < beg[p]) return ion_fail(s, ION_ERR_INVALID_ARG, "pulse %d: end before begin", p);
        if (!std::isfinite(amp[p])) return ion_fail(s, ION_ERR_INVALID_ARG, "pulse %d: amplitude not finite", p);
    }
    // group by cell (stable), offsets per cell
    std::vector<int32_t> order(np);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cell[a] < cell[b]; });
    std::vector<int32_t> off(s->n + 1, 0);
    for (int32_t p = 0; p < np; ++p) off[cell[p] + 1]++;
    for (int32_t i = 0; i < s->n; ++i) off[i + 1] += off[i];
    std::vector<int64_t> b2(np), e2(np);
    std::vector<float> a2(np);
    for (int32_t q = 0; q < np; ++q) {
        b2[q] = beg[order[q]];
        e2[q] = end[order[q]];
        a2[q] = amp[order[q]];
    }
    ION_CK(s, cudaStreamSynchronize(s->st));
    cudaFree(s->d_poff);
    cudaFree(s->d_pbeg);
    cudaFree(s->d_pend);
    cudaFree(s->d_pamp);
    s->d_poff = nullptr;
    s->d_pbeg = s->d_pend = nullptr;
    s->d_pamp = nullptr;
    s->n_pulses = 0;
    ion_drop_graphs(s);
    if (np == 0) return ION_OK;
    cudaError_t e = ion_alloc(&s->d_poff, (s->n + 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = ion_alloc(&s->d_pbeg, np * sizeof(int64_t));
    if (e == cudaSuccess) e = ion_alloc(&s->d_pend, np * sizeof(int64_t));
    if (e == cudaSuccess) e = ion_alloc(&s->d_pamp, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(s->d_poff, off.data(), (s->n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_pbeg, b2.data(), np * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_pend, e2.data(), np * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_pamp, a2.data(), np * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {   // leave no half-built table behind: the kernels would read it
        cudaFree(s->d_poff);
        cudaFree(s->d_pbeg);
        cudaFree(s->d_pend);
        cudaFree(s->d_pamp);
        s->d_poff = nullptr;
        s->d_pbeg = s->d_pend = nullptr;
        s->d_pamp = nullptr;
        return ion_fail(s, e == cudaErrorMemoryAllocation ? ION_ERR_OOM : ION_ERR_CUDA, "ion_set_input: %s",
                        cudaGetErrorString(e));
    }
    s->n_pulses = np;
    return ION_OK;
}

extern "C" ion_status ion_set_input(ion_sim *s, const ion_input *in) {
    if (!s) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_set_input: NULL handle");
    if (!in || in->kind == ION_INPUT_NONE) {
        ion_input none{};
        none.kind = ION_INPUT_PULSES;
        none.n_pulses = 0;
        return install_pulses(s, &none);
    }
    if (in->kind == ION_INPUT_PULSES) return install_pulses(s, in);
    return ion_fail(s, ION_ERR_INVALID_ARG, "ion_set_input: only NONE or PULSES inputs can be installed");
}

// ---- stepping -------------------------------------------------------------------------
StepCommon ion_step_common(ion_sim *s, int k_off, const float *iapp) {
    StepCommon c{};
    c.S.base = s->d_state;
    c.S.stride = s->stride;
    c.n = s->n;
    c.n_pad = s->n_pad;
    c.t_dev = s->d_t;
    c.k_off = k_off;
    c.par = (int32_t)((s->t_enq + k_off) & 1);
    c.vd_fixed = 0;
    c.pulses.off = s->n_pulses > 0 ? s->d_poff : nullptr;   // no table unless one is complete
    c.pulses.begin = s->d_pbeg;
    c.pulses.end = s->d_pend;
    c.pulses.amp = s->d_pamp;
    c.iapp = iapp;
    c.status = s->d_status;
    c.trace = s->d_trace;
    c.trace_stride = s->trace_stride;
    c.trace_cap = s->trace_cap;
    c.pdl = !(s->flags & ION_FLAG_NO_PDL) && !s->pdl_off;
    c.P = s->P;
    return c;
}

// Enqueue one step (offset k_off from the device step counter).
static cudaError_t enqueue_one_step(ion_sim *s, int k_off, const float *iapp) {
    if (s->step_override) return s->step_override(s, k_off, iapp);
    const StepCommon c = ion_step_common(s, k_off, iapp);
    const bool split = (s->flags & ION_FLAG_SPLIT) != 0;
    cudaError_t e = cudaSuccess;
    if (s->kind == ION_DENSE_MATRIX) {
        MatrixArgs a{};
        a.c = c;
        a.W = s->d_W;
        e = launch_matrix_step(a, s->dense_R, s->st);
        s->launches++;
        return e;
    }
    if (s->flags & ION_FLAG_SGJ) {   // linear junctions (SGJ use case)
        if (s->kind == ION_DENSE_UNIFORM) {
            e = launch_sgj_dense_step(c, s->g, s->d_sgj, s->st);
            s->launches += s->lps;
        } else {
            // the compact CSR kernels with the linear term where the network has 16-bit
            // columns (staged or not, as for the exponential junction), else eight lanes
            // per row over the 32-bit columns
            const bool staged = s->csr_staged == 1 && !split;
            CsrArgs a{};
            a.c = c;
            ion_csr_fill(s, a, staged);
            if (a.col16 != nullptr && !split) {
                a.lin = 1;
                a.fuse = 1;
                e = staged ? launch_csr_chunk_step(a, s->csr_chunk_SW, s->csr_chunk_rows, s->d_mid, s->n_chunks, false,
                                                   s->st)
                           : launch_csr_step(a, s->csr_SW, s->csr_rows, s->st);
            } else {
                a.col16 = nullptr;
                e = launch_sgj_csr_step(a, s->st);
            }
            s->launches++;
        }
        return e;
    }
    if (s->kind == ION_DENSE_UNIFORM) {
        DenseArgs a{};
        a.c = c;
        a.g = s->g;
        a.kahan = 1;
        a.fuse = split ? 0 : 1;
        a.ic_out = s->d_ic;
        a.vd_in = nullptr;
        e = launch_dense_step(a, s->dense_R, s->dense_W, s->dense_GJ, s->st);
        s->launches++;
        if (e == cudaSuccess && split) {
            CellArgs ca{c, s->d_ic, s->d_cellp};
            e = launch_cell_step(ca, s->st);
            s->launches++;
        }
    } else if (s->kind == ION_CSR && s->d_rev) {   // half-work: upper pass, then lower pass + update
        CsrArgs a{};
        a.c = c;
        a.row_ptr = s->d_rowptr;
        a.col = s->d_col;
        a.w = s->d_w;
        a.g = s->g;
        a.fuse = 1;
        e = launch_csr_half_step(a, s->csr_SW, s->csr_rows, s->d_split, s->d_rev, s->d_slot, s->d_icu, s->st);
        s->launches += 2;
    } else if (s->kind == ION_CSR) {
        CsrArgs a{};
        a.c = c;
        ion_csr_fill(s, a, s->csr_staged == 1 && !split);
        a.fuse = split ? 0 : 1;
        a.ic_out = s->d_ic;
        a.vd_in = nullptr;
        if (s->csr_staged == 1 && !split)
            e = launch_csr_chunk_step(a, s->csr_chunk_SW, s->csr_chunk_rows, s->d_mid, s->n_chunks, false, s->st);
        else
            e = launch_csr_step(a, s->csr_SW, s->csr_rows, s->st);
        s->launches++;
        if (e == cudaSuccess && split) {
            CellArgs ca{c, s->d_ic, s->d_cellp};
            e = launch_cell_step(ca, s->st);
            s->launches++;
        }
    } else {
        CellArgs ca{c, nullptr, s->d_cellp};
        e = launch_cell_step(ca, s->st);
        s->launches++;
    }
    return e;
}

// Enqueue k steps directly (no graph) followed by the device counter advance.
static cudaError_t enqueue_steps_direct(ion_sim *s, int64_t k, const float *iapp_base) {
    int64_t done = 0;
    while (done < k) {
        const int64_t chunk = std::min<int64_t>(k - done, 1 << 20);
        for (int64_t j = 0; j < chunk; ++j) {
            const float *iapp = iapp_base ? iapp_base + (done + j) * (int64_t)s->n : nullptr;
            cudaError_t e = enqueue_one_step(s, (int)j, iapp);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = launch_advance(s->d_t, chunk, s->st);
        s->launches++;
        if (e != cudaSuccess) return e;
        s->t_enq += chunk;
        done += chunk;
    }
    return cudaSuccess;
}

static ion_status build_graph_once(ion_sim *s) {
    const int K = s->graph_steps;
    cudaGraph_t g = nullptr;
    const int64_t launches0 = s->launches;
    ION_CK(s, cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < K && e == cudaSuccess; ++j) e = enqueue_one_step(s, j, nullptr);
    if (e == cudaSuccess) e = launch_advance(s->d_t, K, s->st);
    cudaError_t e2 = cudaStreamEndCapture(s->st, &g);
    s->launches = launches0;
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return ion_fail(s, ION_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t &gx = s->gexec[s->t_enq & 1];   // its launches take the parity of the current step
    e = cudaGraphInstantiate(&gx, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        gx = nullptr;
        return ion_fail(s, ION_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    s->graph_launches = (int64_t)K * s->launches_per_step() + 1;   // + the counter advance
    return ION_OK;
}

// Capture the K-step graph; if a capture with programmatic launches is refused, capture
// again with ordinary launches (and keep them for this handle).
static ion_status build_graph(ion_sim *s) {
    ion_status st = build_graph_once(s);
    if (st == ION_OK || (s->flags & ION_FLAG_NO_PDL) || s->pdl_off) return st;
    (void)cudaGetLastError();
    s->pdl_off = true;
    return build_graph_once(s);
}

extern "C" ion_status ion_step(ion_sim *s, int64_t n_steps, const ion_input *input) {
    if (!s) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_step: NULL handle");
    if (n_steps < 0) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_step: negative n_steps");
    if (n_steps == 0) return ION_OK;
    const float *iapp = nullptr;
    if (input && input->kind == ION_INPUT_PULSES) {
        ion_status st = install_pulses(s, input);
        if (st != ION_OK) return st;
    } else if (input && input->kind == ION_INPUT_DENSE) {
        if (!input->dense) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_step: NULL dense input");
        const int64_t cnt = n_steps * (int64_t)s->n;
        if (input->mem == ION_DEVICE) {
            iapp = input->dense;
        } else {
            if (cnt > s->iapp_cap) {
                ION_CK(s, cudaStreamSynchronize(s->st));
                cudaFree(s->d_iapp);
                s->d_iapp = nullptr;
                s->iapp_cap = 0;
                ION_CK(s, ion_alloc(&s->d_iapp, (size_t)cnt * sizeof(float)));
                s->iapp_cap = cnt;
            }
            ION_CK(s, cudaMemcpyAsync(s->d_iapp, input->dense, (size_t)cnt * sizeof(float), cudaMemcpyHostToDevice, s->st));
            iapp = s->d_iapp;
        }
    } else if (input && input->kind != ION_INPUT_NONE) {
        return ion_fail(s, ION_ERR_INVALID_ARG, "ion_step: unknown input kind %d", input->kind);
    } else if (input && input->kind == ION_INPUT_NONE && s->n_pulses > 0) {
        ion_status st = ion_set_input(s, nullptr);
        if (st != ION_OK) return st;
    }
    if (s->prepare_hook) {
        ion_status st = s->prepare_hook(s);
        if (st != ION_OK) return st;
    }
    // a pending asynchronous trace copy still reads ring slots: steps that would write the
    // sample taking the first of them wait for the copy
    if (s->copy_pending && s->trace_stride > 0 && (s->t + n_steps) / s->trace_stride > s->copy_guard_sample) {
        ION_CK(s, cudaStreamWaitEvent(s->st, s->ev_copied, 0));
        s->copy_guard_sample = INT64_MAX;   // ordered after the copy; the host still waits in ion_trace_wait
    }
    if (s->run_override && iapp == nullptr) {
        ion_status st = s->run_override(s, n_steps, iapp);
        if (st != ION_OK) return st;
        s->t += n_steps;
        return ION_OK;
    }
    int64_t left = n_steps;
    s->t_enq = s->t;
    const bool graphs = !(s->flags & ION_FLAG_NO_GRAPH) && iapp == nullptr && !s->no_graph;
    while (graphs && left >= s->graph_steps) {
        const int p = (int)(s->t_enq & 1);
        if (!s->gexec[p]) {
            ion_status st = build_graph(s);
            if (st != ION_OK) return st;
        }
        ION_CK(s, cudaGraphLaunch(s->gexec[p], s->st));
        s->launches += s->graph_launches;
        left -= s->graph_steps;
        s->t_enq += s->graph_steps;
    }
    if (left > 0) {
        const float *base = iapp ? iapp + (n_steps - left) * (int64_t)s->n : nullptr;
        cudaError_t e = enqueue_steps_direct(s, left, base);
        if (e != cudaSuccess) return ion_fail(s, ION_ERR_CUDA, "ion_step: launch: %s", cudaGetErrorString(e));
    }
    s->t += n_steps;
    return ION_OK;
}

// ---- synchronisation and state I/O ----------------------------------------------------
extern "C" ion_status ion_sync(ion_sim *s) {
    if (!s) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_sync: NULL handle");
    ION_CK(s, cudaStreamSynchronize(s->st));
    uint32_t st = 0;
    ION_CK(s, cudaMemcpy(&st, s->d_status, sizeof st, cudaMemcpyDeviceToHost));
    s->sticky |= st;
    if (s->sticky & ST_TIMEOUT) return ion_fail(s, ION_ERR_TIMEOUT, "a bounded device wait timed out");
    if (s->sticky & ST_NONFINITE) return ion_fail(s, ION_ERR_NONFINITE, "non-finite voltage or [Ca] in the state");
    if (s->sticky & ST_SLOT)
        return ion_fail(s, ION_ERR_CUDA, "the device step counter and the host's step count disagree");
    return ION_OK;
}

float *ion_field_ptr(ion_sim *s, int32_t field) {
    if (field == ION_V_DEND) return s->d_state + ((s->t & 1) ? 19 : 0) * s->stride;
    return s->d_state + (int64_t)field * s->stride;
}

extern "C" ion_status ion_state_device_ptr(ion_sim *s, int32_t field, float **out) {
    if (!s || !out || field < 0 || field >= NF) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_state_device_ptr: bad arguments");
    if (s->d_map) return ion_fail(s, ION_ERR_UNSUPPORTED, "ion_state_device_ptr: not available for batches");
    if (s->state_sync_hook) {
        ion_status st = s->state_sync_hook(s);
        if (st != ION_OK) return st;
    }
    *out = ion_field_ptr(s, field);
    return ION_OK;
}

extern "C" ion_status ion_read_state(ion_sim *s, int32_t field, float *out, int64_t count) {
    if (!s || !out) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_read_state: NULL argument");
    if (field != ION_FIELD_ALL && (field < 0 || field >= NF))
        return ion_fail(s, ION_ERR_INVALID_ARG, "ion_read_state: field %d out of range", field);
    const int64_t need = field == ION_FIELD_ALL ? (int64_t)NF * s->n_user : s->n_user;
    if (count != need) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_read_state: count %lld, expected %lld", (long long)count, (long long)need);
    if (s->state_sync_hook) {
        ion_status st = s->state_sync_hook(s);
        if (st != ION_OK) return st;
    }
    const ion_status st = ion_sync(s);
    if (st != ION_OK && st != ION_ERR_NONFINITE && st != ION_ERR_TIMEOUT) return st;
    if (s->d_map) {
        const ion_status st2 = ion_batch_read(s, field, out);
        return st2 != ION_OK ? st2 : st;
    }
    if (field == ION_FIELD_ALL) {
        ION_CK(s, cudaMemcpy2D(out, s->n * sizeof(float), s->d_state, s->stride * sizeof(float), s->n * sizeof(float), NF,
                               cudaMemcpyDeviceToHost));
        ION_CK(s, cudaMemcpy(out, ion_field_ptr(s, ION_V_DEND), s->n * sizeof(float), cudaMemcpyDeviceToHost));
    } else {
        ION_CK(s, cudaMemcpy(out, ion_field_ptr(s, field), s->n * sizeof(float), cudaMemcpyDeviceToHost));
    }
    return st;
}

extern "C" ion_status ion_write_state(ion_sim *s, int32_t field, const float *in, int64_t count) {
    if (!s || !in) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_write_state: NULL argument");
    if (field != ION_FIELD_ALL && (field < 0 || field >= NF))
        return ion_fail(s, ION_ERR_INVALID_ARG, "ion_write_state: field %d out of range", field);
    const int64_t need = field == ION_FIELD_ALL ? (int64_t)NF * s->n_user : s->n_user;
    if (count != need) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_write_state: count %lld, expected %lld", (long long)count, (long long)need);
    if (s->state_sync_hook) {
        ion_status st = s->state_sync_hook(s);
        if (st != ION_OK) return st;
    }
    if (s->d_map) {
        ION_CK(s, cudaStreamSynchronize(s->st));
        return ion_batch_write(s, field, in);
    }
    if (field == ION_FIELD_ALL) {
        ION_CK(s, cudaMemcpy2DAsync(s->d_state, s->stride * sizeof(float), in, s->n * sizeof(float), s->n * sizeof(float), NF,
                                    cudaMemcpyHostToDevice, s->st));
        if (s->t & 1)
            ION_CK(s, cudaMemcpyAsync(ion_field_ptr(s, ION_V_DEND), in, s->n * sizeof(float), cudaMemcpyHostToDevice, s->st));
    } else {
        ION_CK(s, cudaMemcpyAsync(ion_field_ptr(s, field), in, s->n * sizeof(float), cudaMemcpyHostToDevice, s->st));
    }
    ION_CK(s, cudaStreamSynchronize(s->st));
    if (s->state_load_hook) return s->state_load_hook(s);
    return ION_OK;
}

extern "C" ion_status ion_set_step_count(ion_sim *s, int64_t t) {
    if (!s || t < 0) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_set_step_count: bad arguments");
    if (s->state_sync_hook) {
        ion_status st = s->state_sync_hook(s);
        if (st != ION_OK) return st;
    }
    ION_CK(s, cudaStreamSynchronize(s->st));
    if ((t & 1) != (s->t & 1))   // keep V_dend in the slot the kernels read at step t
        ION_CK(s, cudaMemcpy(s->d_state + ((t & 1) ? 19 : 0) * s->stride, ion_field_ptr(s, ION_V_DEND),
                             s->n * sizeof(float), cudaMemcpyDeviceToDevice));
    ION_CK(s, cudaMemcpy(s->d_t, &t, sizeof t, cudaMemcpyHostToDevice));
    s->t = t;
    if (s->d_trace) s->trace_read = t / s->trace_stride;
    if (s->state_load_hook) return s->state_load_hook(s);
    return ION_OK;
}

// ---- V_axon trace -------------------------------------------------------------------------
extern "C" ion_status ion_set_trace(ion_sim *s, int32_t stride, int32_t capacity) {
    if (!s || stride < 0 || capacity < 0) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_set_trace: bad arguments");
    ION_CK(s, cudaStreamSynchronize(s->st));
    if (s->copy_st) ION_CK(s, cudaStreamSynchronize(s->copy_st));
    s->copy_pending = false;
    cudaFree(s->d_trace);
    s->d_trace = nullptr;
    s->trace_stride = 0;
    s->trace_cap = 0;
    ion_drop_graphs(s);
    if (stride == 0 || capacity == 0) return ION_OK;
    ION_CK(s, ion_alloc(&s->d_trace, (size_t)capacity * s->n * sizeof(float)));
    s->trace_stride = stride;
    s->trace_cap = capacity;
    s->trace_read = s->t / stride;
    return ION_OK;
}

extern "C" ion_status ion_read_trace(ion_sim *s, float *out, int64_t max_samples, int64_t *n_written) {
    if (!s || !n_written) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_read_trace: NULL argument");
    *n_written = 0;
    if (!s->d_trace) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_read_trace: tracing is off");
    if (s->state_sync_hook) {
        ion_status st0 = s->state_sync_hook(s);
        if (st0 != ION_OK) return st0;
    }
    const ion_status st = ion_sync(s);
    if (st != ION_OK && st != ION_ERR_NONFINITE && st != ION_ERR_TIMEOUT) return st;
    const int64_t produced = s->t / s->trace_stride;
    int64_t first = s->trace_read;
    if (produced - first > s->trace_cap) first = produced - s->trace_cap;   // overwritten samples are lost
    const int64_t avail = produced - first;
    const int64_t take = std::min(avail, max_samples);
    if (take > 0 && !out) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_read_trace: NULL out");
    std::vector<float> tmp(s->d_map ? (size_t)s->n : 0);
    for (int64_t k = 0; k < take; ++k) {
        const int64_t slot = (first + k) % s->trace_cap;
        if (!s->d_map) {
            ION_CK(s, cudaMemcpy(out + k * s->n, s->d_trace + slot * s->n, s->n * sizeof(float), cudaMemcpyDeviceToHost));
        } else {   // batch: compact the padded sample into the user numbering
            ION_CK(s, cudaMemcpy(tmp.data(), s->d_trace + slot * s->n, s->n * sizeof(float), cudaMemcpyDeviceToHost));
            for (int64_t j = 0; j < s->n_user; ++j) out[k * s->n_user + j] = tmp[(size_t)ion_batch_map_cell(s, j)];
        }
    }
    s->trace_read = first + take;
    *n_written = take;
    return st;
}

// Asynchronous drain of the V_axon ring: the copy runs on the handle's copy stream after
// the steps already enqueued, so later steps overlap it (the paper's GPU design overlaps
// the transfer of step t with the computation of step t + 1, Sec. 2.4.3).  Steps that
// would overwrite a slot the pending copy still reads wait for it first.
extern "C" ion_status ion_read_trace_async(ion_sim *s, float *out, int64_t max_samples, int64_t *n_queued) {
    if (!s || !n_queued) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_read_trace_async: NULL argument");
    *n_queued = 0;
    if (!s->d_trace) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_read_trace_async: tracing is off");
    if (s->d_map) return ion_fail(s, ION_ERR_UNSUPPORTED, "ion_read_trace_async: not for batches (use ion_read_trace)");
    if (max_samples < 0) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_read_trace_async: negative max_samples");
    const int64_t produced = s->t / s->trace_stride;
    int64_t first = s->trace_read;
    if (produced - first > s->trace_cap) first = produced - s->trace_cap;   // overwritten samples are lost
    const int64_t take = std::min(produced - first, max_samples);
    if (take > 0 && !out) return ion_fail(s, ION_ERR_INVALID_ARG, "ion_read_trace_async: NULL out");
    if (!s->copy_st) {
        ION_CK(s, cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking));
        ION_CK(s, cudaEventCreateWithFlags(&s->ev_ready, cudaEventDisableTiming));
        ION_CK(s, cudaEventCreateWithFlags(&s->ev_copied, cudaEventDisableTiming));
    }
    if (take > 0) {
        ION_CK(s, cudaEventRecord(s->ev_ready, s->st));
        ION_CK(s, cudaStreamWaitEvent(s->copy_st, s->ev_ready, 0));
        const int64_t slot0 = first % s->trace_cap;
        const int64_t k1 = std::min(take, s->trace_cap - slot0);    // up to the ring's end, then from slot 0
        ION_CK(s, cudaMemcpyAsync(out, s->d_trace + slot0 * s->n, (size_t)(k1 * s->n) * sizeof(float),
                                  cudaMemcpyDeviceToHost, s->copy_st));
        if (take > k1)
            ION_CK(s, cudaMemcpyAsync(out + k1 * s->n, s->d_trace, (size_t)((take - k1) * s->n) * sizeof(float),
                                      cudaMemcpyDeviceToHost, s->copy_st));
        ION_CK(s, cudaEventRecord(s->ev_copied, s->copy_st));
        s->copy_pending = true;
        s->copy_guard_sample = first + s->trace_cap;
    }
    s->trace_read = first + take;
    *n_queued = take;
    return ION_OK;
}

extern "C" ion_status ion_trace_wait(ion_sim *s) {
    if (!s) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_trace_wait: NULL handle");
    if (s->copy_pending) {
        ION_CK(s, cudaEventSynchronize(s->ev_copied));
        s->copy_pending = false;
    }
    return ION_OK;
}

// ---- single-launch primitives ---------------------------------------------------------------
extern "C" ion_status ion_gj_dense(const float *vdend, int32_t n, float g_c, float *ic, int32_t kahan, void *stream) {
    if (!vdend || !ic || n < 1) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_gj_dense: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const int n_pad = (int)round_up(n, PAD_J);
    float *pad = nullptr;
    ION_CK(nullptr, cudaMallocAsync(&pad, (size_t)n_pad * sizeof(float), st));
    cudaError_t e = cudaMemcpyAsync(pad, vdend, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = launch_fill(pad + n, PAD_VOLT, n_pad - n, st);
    int R, W, GJ;
    ion_choose_dense_shape(n, num_sms(), &R, &W, &GJ);
    if (e == cudaSuccess) e = prepare_dense_step(R, W, GJ, n_pad);
    if (e == cudaSuccess) {
        DenseArgs a{};
        a.c.n = n;
        a.c.n_pad = n_pad;
        a.g = g_c;
        a.kahan = kahan ? 1 : 0;
        a.fuse = 0;
        a.ic_out = ic;
        a.vd_in = pad;
        e = launch_dense_step(a, R, W, GJ, st);
    }
    cudaError_t e2 = cudaFreeAsync(pad, st);
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "ion_gj_dense: %s", cudaGetErrorString(e));
    if (e2 != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "ion_gj_dense: %s", cudaGetErrorString(e2));
    return ION_OK;
}

extern "C" ion_status ion_gj_csr(const float *vdend, int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                 const float *w, float g_c, float *ic, void *stream) {
    if (!vdend || !ic || !row_ptr || n < 1) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_gj_csr: bad arguments");
    CsrArgs a{};
    a.c.n = n;
    a.row_ptr = row_ptr;
    a.col = col_idx;
    a.w = w;
    a.g = g_c;
    a.fuse = 0;
    a.ic_out = ic;
    a.vd_in = vdend;
    // mean degree is unknown without reading row_ptr[n]; lanes per row = 8 suits 10..100
    cudaError_t e = launch_csr_step(a, 8, 256, (cudaStream_t)stream);
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "ion_gj_csr: %s", cudaGetErrorString(e));
    return ION_OK;
}

extern "C" ion_status ion_cell_update(float *state, int32_t n, const float *ic, const float *iapp, const ion_model *model,
                                      double dt_ms, void *stream) {
    if (!state || n < 1) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_cell_update: bad arguments");
    ion_model m;
    if (model) m = *model;
    else ion_model_default(&m);
    if (!model_valid(m)) return ion_fail(nullptr, ION_ERR_INVALID_ARG, "ion_cell_update: invalid model table");
    const double dt = dt_ms > 0 ? dt_ms : 0.05;
    CellArgs a{};
    a.c.S.base = state;
    a.c.S.stride = n;
    a.c.n = n;
    a.c.n_pad = n;
    a.c.vd_fixed = 1;
    a.c.P = ion_model_to_f32(m, dt);
    a.c.iapp = iapp;
    a.ic = ic;
    // the status word is not reported by this primitive: point it at a private word
    static uint32_t *d_dummy = nullptr;
    if (!d_dummy) ION_CK(nullptr, ion_alloc(&d_dummy, sizeof(uint32_t)));
    a.c.status = d_dummy;
    cudaError_t e = launch_cell_step(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return ion_fail(nullptr, ION_ERR_CUDA, "ion_cell_update: %s", cudaGetErrorString(e));
    return ION_OK;
}
