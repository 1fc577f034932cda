// ion_model.cuh -- FP32 device model of the three-compartment inferior-olive cell.
//
// Paper: Smaragdos et al., "BrainFrame" (arXiv 1612.01501), Sec. 2.2 "The InfOli
// Workload": each cell has a dendrite (with the gap junctions), a soma and an axon
// whose voltage is the cell output; every new state depends only on the previous
// state, the previous dendritic voltages of its partners and the evoked input, and all
// parts are updated concurrently with a 50 us step.  We read "concurrently" as pure
// explicit Euler: every right-hand side below takes step-t values.
//
// The cell equations are the published three-compartment IO cell the paper cites
// (De Gruijl et al. 2012; the paper does not print them): dendrite high-threshold Ca
// (r^2), Ca-activated K (s), h-current (q), leak and a [Ca] pool; soma low-threshold
// Ca (k^3 l), Na (m_inf^3 h), delayed-rectifier K (n^4), voltage-gated K (x^4), leak;
// axon Na (m_inf^3 h), K (x^4), leak; ohmic dendrite-soma and soma-axon coupling
// scaled by the compartments' area shares p1, p2.
//
// Arithmetic: FP32 throughout; exponentials are 2^(x log2 e) on the SFU
// (ex2.approx.ftz) and divisions are multiplications by an SFU reciprocal
// (rcp.approx.ftz).  Removable singularities z / (e^z - 1) use a 4th-order Taylor
// expansion for |z| < 0.05.
#pragma once
#include <cstdint>

namespace ion {

constexpr int NF = 19;
enum Field {
    F_VDEND = 0, F_VSOMA, F_VAXON, F_CA, F_R, F_S, F_Q, F_K, F_L, F_MS, F_HS, F_NS, F_XS,
    F_MA, F_HA, F_XA, F_GCAL, F_ICAH, F_IC
};
constexpr int NG = 12;
enum Gate { G_R = 0, G_S, G_Q, G_K, G_L, G_MS, G_HS, G_NS, G_XS, G_MA, G_HA, G_XA };

// FP32 constants handed to every kernel by value (they land in the constant bank).
struct ModelF {
    float g_ds;    // g_int / (1 - p1): dendrite side of the dendrite-soma junction
    float g_sd;    // g_int / p1:       soma side of the dendrite-soma junction
    float g_sa;    // g_int / (1 - p2): soma side of the soma-axon junction
    float g_as;    // g_int / p2:       axon side of the soma-axon junction
    float gCaH, gKCa, gh, gld;
    float gNas, gKdrs, gKs, gls;
    float gNaa, gKa, gla;
    float VNa, VK, VCa, Vh, VL;
    float dt_cm;   // dt / C_m
    float dt;      // dt (gates and [Ca])
    float ca_in, ca_out;
};
// A cell may own the first NCELLP members of ModelF (g_ds ... VL): Table "reqs" gives
// every neuron its own conductances.
constexpr int NCELLP = 20;

// The model constants of cell i: the shared ones with the cell's own first NCELLP members
// (row k of cp, stride floats per row).
__device__ __forceinline__ ModelF cell_model(const ModelF &P, const float *__restrict__ cp, int64_t stride,
                                             int64_t i) {
    ModelF q = P;
    const float *c = cp + i;
    q.g_ds = c[0 * stride];
    q.g_sd = c[1 * stride];
    q.g_sa = c[2 * stride];
    q.g_as = c[3 * stride];
    q.gCaH = c[4 * stride];
    q.gKCa = c[5 * stride];
    q.gh = c[6 * stride];
    q.gld = c[7 * stride];
    q.gNas = c[8 * stride];
    q.gKdrs = c[9 * stride];
    q.gKs = c[10 * stride];
    q.gls = c[11 * stride];
    q.gNaa = c[12 * stride];
    q.gKa = c[13 * stride];
    q.gla = c[14 * stride];
    q.VNa = c[15 * stride];
    q.VK = c[16 * stride];
    q.VCa = c[17 * stride];
    q.Vh = c[18 * stride];
    q.VL = c[19 * stride];
    return q;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// e^x = 2^(x log2 e)
__device__ __forceinline__ float expf_sfu(float x) { return ex2_approx(x * 1.4426950408889634f); }

// z / (e^z - 1), continuous at 0 (value 1)
__device__ __forceinline__ float z_over_expm1(float z) {
    if (fabsf(z) < 0.05f) return 1.0f + z * (-0.5f + z * (1.0f / 12.0f - z * z * (1.0f / 720.0f)));
    return z * rcp_approx(expf_sfu(z) - 1.0f);
}
// 1 / (1 + e^{-(V - vh) / k}) with the inverse slope precomputed
__device__ __forceinline__ float rise(float V, float vh, float inv_k) {
    return rcp_approx(1.0f + expf_sfu((vh - V) * inv_k));
}
// 1 / (1 + e^{(V - vh) / k})
__device__ __forceinline__ float fall(float V, float vh, float inv_k) {
    return rcp_approx(1.0f + expf_sfu((V - vh) * inv_k));
}

// ---- rate functions: steady state xinf and the rate 1/tau -----------------------
// (the update needs dt / tau, so the reciprocal of tau is what is produced)
struct Rate { float xinf, inv_tau; };

__device__ __forceinline__ Rate rate_r(float V) {  // dendrite high-threshold Ca
    float a = 1.7f * rcp_approx(1.0f + expf_sfu((5.0f - V) * (1.0f / 13.9f)));
    float b = 0.1f * z_over_expm1((V + 8.5f) * 0.2f);   // 0.02 (V+8.5) / (e^{(V+8.5)/5} - 1)
    float inv_ab = rcp_approx(a + b);
    return {a * inv_ab, (a + b) * 0.2f};                 // tau = 5 / (a + b)
}
__device__ __forceinline__ Rate rate_s(float ca) {  // dendrite Ca-activated K
    float a = fminf(2.0e-5f * ca, 0.01f);
    float ab = a + 0.015f;
    return {a * rcp_approx(ab), ab};
}
__device__ __forceinline__ Rate rate_q(float V) {  // dendrite h-current
    float xinf = fall(V, -80.0f, 0.25f);
    float inv_tau = expf_sfu(-0.086f * V - 14.6f) + expf_sfu(0.070f * V - 1.87f);
    return {xinf, inv_tau};
}
__device__ __forceinline__ Rate rate_k(float V) {  // soma low-threshold Ca activation, tau = 1
    return {rise(V, -61.0f, 1.0f / 4.2f), 1.0f};
}
__device__ __forceinline__ Rate rate_l(float V) {  // soma low-threshold Ca inactivation
    float xinf = fall(V, -85.5f, 1.0f / 8.5f);
    float tau = 20.0f * expf_sfu((V + 160.0f) * (1.0f / 30.0f)) *
                    rcp_approx(1.0f + expf_sfu((V + 84.0f) * (1.0f / 7.3f))) + 35.0f;
    return {xinf, rcp_approx(tau)};
}
__device__ __forceinline__ float minf_na(float V) { return rise(V, -30.0f, 1.0f / 5.5f); }
__device__ __forceinline__ Rate rate_hs(float V) {  // soma Na inactivation, tau = 3 e^{-(V+40)/33}
    return {fall(V, -70.0f, 1.0f / 5.8f), (1.0f / 3.0f) * expf_sfu((V + 40.0f) * (1.0f / 33.0f))};
}
__device__ __forceinline__ Rate rate_ns(float V) {  // soma delayed-rectifier K
    float tau = 5.0f + 47.0f * expf_sfu((V + 50.0f) * (1.0f / 900.0f));
    return {rise(V, -3.0f, 0.1f), rcp_approx(tau)};
}
__device__ __forceinline__ Rate rate_x(float V) {  // soma/axon voltage-gated K
    float a = 1.3f * z_over_expm1(-(V + 25.0f) * 0.1f);  // 0.13 (V+25) / (1 - e^{-(V+25)/10})
    float b = 1.69f * expf_sfu(-0.0125f * (V + 35.0f));
    float ab = a + b;
    return {a * rcp_approx(ab), ab};
}
__device__ __forceinline__ Rate rate_ha(float V) {  // axon Na inactivation, tau = 1.5 e^{-(V+40)/33}
    return {fall(V, -60.0f, 1.0f / 5.8f), (1.0f / 1.5f) * expf_sfu((V + 40.0f) * (1.0f / 33.0f))};
}

// ---- one cell, one explicit-Euler step -------------------------------------------
struct Cell {   // the 15 words the update reads
    float vd, vs, va, ca, r, s, q, k, l, hs, ns, xs, ha, xa, gcal;
};
struct CellNext {  // the 18 words it writes (g_CaL is constant)
    float vd, vs, va, ca, r, s, q, k, l, ms, hs, ns, xs, ma, ha, xa, icah, ic;
};

// x + dt (xinf - x) / tau
__device__ __forceinline__ float relax(float x, Rate g, float dt) { return fmaf(dt * g.inv_tau, g.xinf - x, x); }

// Rates of one cell's gates (the m_s / m_a entries only use xinf).
struct CellRates {
    Rate r, s, q, k, l, ms, hs, ns, xs, ma, ha, xa;
};

__device__ __forceinline__ CellRates exact_rates(const Cell &c) {
    CellRates g;
    g.r = rate_r(c.vd);
    g.s = rate_s(c.ca);
    g.q = rate_q(c.vd);
    g.k = rate_k(c.vs);
    g.l = rate_l(c.vs);
    g.ms = Rate{minf_na(c.vs), 0.0f};
    g.hs = rate_hs(c.vs);
    g.ns = rate_ns(c.vs);
    g.xs = rate_x(c.vs);
    g.ma = Rate{minf_na(c.va), 0.0f};
    g.ha = rate_ha(c.va);
    g.xa = rate_x(c.va);
    return g;
}

// ---- the three compartment voltages (and [Ca]) of one explicit-Euler step ---------
// Each function computes its outputs from the step-t cell alone.  The single-thread step
// below and the split update (one cell's outputs spread over several threads, see
// ion_kernels.cuh) both call them, so either way a cell gets the same bits.
struct DendNext { float vd, ca, icah; };
__device__ __forceinline__ DendNext dend_step(const ModelF &P, const Cell &c, float ic, float iapp) {
    DendNext o;
    const float I_CaH = P.gCaH * c.r * c.r * (c.vd - P.VCa);
    const float I_KCa = P.gKCa * c.s * (c.vd - P.VK);
    const float I_h = P.gh * c.q * (c.vd - P.Vh);
    const float I_ld = P.gld * (c.vd - P.VL);
    const float I_ds = P.g_ds * (c.vd - c.vs);
    o.vd = fmaf(P.dt_cm, iapp - I_CaH - I_KCa - I_h - I_ld - I_ds - ic, c.vd);
    o.ca = fmaf(P.dt, -P.ca_in * I_CaH - P.ca_out * c.ca, c.ca);
    o.icah = I_CaH;
    return o;
}
// ms = m_inf(V_soma) of step t
__device__ __forceinline__ float soma_step(const ModelF &P, const Cell &c, float ms) {
    const float k3 = c.k * c.k * c.k;
    const float n2 = c.ns * c.ns, x2 = c.xs * c.xs;
    const float I_CaL = c.gcal * k3 * c.l * (c.vs - P.VCa);
    const float I_Nas = P.gNas * ms * ms * ms * c.hs * (c.vs - P.VNa);
    const float I_Kdr = P.gKdrs * n2 * n2 * (c.vs - P.VK);
    const float I_Ks = P.gKs * x2 * x2 * (c.vs - P.VK);
    const float I_ls = P.gls * (c.vs - P.VL);
    const float I_sd = P.g_sd * (c.vs - c.vd);
    const float I_sa = P.g_sa * (c.vs - c.va);
    return fmaf(-P.dt_cm, I_CaL + I_Nas + I_Kdr + I_Ks + I_ls + I_sd + I_sa, c.vs);
}
// ma = m_inf(V_axon) of step t
__device__ __forceinline__ float axon_step(const ModelF &P, const Cell &c, float ma) {
    const float xa2 = c.xa * c.xa;
    const float I_Naa = P.gNaa * ma * ma * ma * c.ha * (c.va - P.VNa);
    const float I_Ka = P.gKa * xa2 * xa2 * (c.va - P.VK);
    const float I_la = P.gla * (c.va - P.VL);
    const float I_as = P.g_as * (c.va - c.vs);
    return fmaf(-P.dt_cm, I_Naa + I_Ka + I_la + I_as, c.va);
}

// One explicit-Euler step of one cell given its gates' rates (exact or learned).
__device__ __forceinline__ CellNext cell_step_rates(const ModelF &P, const Cell &c, float ic, float iapp,
                                                    const CellRates &g) {
    CellNext o;
    const float dt = P.dt;
    const DendNext d = dend_step(P, c, ic, iapp);
    o.vd = d.vd;
    o.ca = d.ca;
    o.icah = d.icah;
    o.ic = ic;
    o.r = relax(c.r, g.r, dt);
    o.s = relax(c.s, g.s, dt);
    o.q = relax(c.q, g.q, dt);
    o.ms = g.ms.xinf;
    o.vs = soma_step(P, c, o.ms);
    o.k = relax(c.k, g.k, dt);
    o.l = relax(c.l, g.l, dt);
    o.hs = relax(c.hs, g.hs, dt);
    o.ns = relax(c.ns, g.ns, dt);
    o.xs = relax(c.xs, g.xs, dt);
    o.ma = g.ma.xinf;
    o.va = axon_step(P, c, o.ma);
    o.ha = relax(c.ha, g.ha, dt);
    o.xa = relax(c.xa, g.xa, dt);
    return o;
}

__device__ __forceinline__ CellNext cell_step(const ModelF &P, const Cell &c, float ic, float iapp) {
    return cell_step_rates(P, c, ic, iapp, exact_rates(c));
}

// ---- SoA access -----------------------------------------------------------------
// The state lives in one buffer of 19 * stride floats (field f at f * stride); V_dend
// is double-buffered: the step-t value is read from vd_cur and the step-(t+1) value is
// written to vd_next (the F_VDEND slot of the main buffer is not used by the kernels).
struct StateView {
    float *base;        // 19 * stride floats
    int64_t stride;     // >= n, multiple of 4
    __device__ __forceinline__ float *f(int field) const { return base + field * stride; }
};

// The 15 words of cell i, V_dend given (persistent launches read it from a staged copy)
__device__ __forceinline__ Cell load_cell(const StateView &S, const float *vd_cur, int64_t i, float vd) {
    (void)vd_cur;
    Cell c;
    c.vd = vd;
    c.vs = S.f(F_VSOMA)[i];
    c.va = S.f(F_VAXON)[i];
    c.ca = S.f(F_CA)[i];
    c.r = S.f(F_R)[i];
    c.s = S.f(F_S)[i];
    c.q = S.f(F_Q)[i];
    c.k = S.f(F_K)[i];
    c.l = S.f(F_L)[i];
    c.hs = S.f(F_HS)[i];
    c.ns = S.f(F_NS)[i];
    c.xs = S.f(F_XS)[i];
    c.ha = S.f(F_HA)[i];
    c.xa = S.f(F_XA)[i];
    c.gcal = S.f(F_GCAL)[i];
    return c;
}

__device__ __forceinline__ Cell load_cell(const StateView &S, const float *vd_cur, int64_t i) {
    Cell c;
    c.vd = vd_cur[i];
    c.vs = S.f(F_VSOMA)[i];
    c.va = S.f(F_VAXON)[i];
    c.ca = S.f(F_CA)[i];
    c.r = S.f(F_R)[i];
    c.s = S.f(F_S)[i];
    c.q = S.f(F_Q)[i];
    c.k = S.f(F_K)[i];
    c.l = S.f(F_L)[i];
    c.hs = S.f(F_HS)[i];
    c.ns = S.f(F_NS)[i];
    c.xs = S.f(F_XS)[i];
    c.ha = S.f(F_HA)[i];
    c.xa = S.f(F_XA)[i];
    c.gcal = S.f(F_GCAL)[i];
    return c;
}

__device__ __forceinline__ void store_cell(const StateView &S, float *vd_next, int64_t i, const CellNext &o) {
    vd_next[i] = o.vd;
    S.f(F_VSOMA)[i] = o.vs;
    S.f(F_VAXON)[i] = o.va;
    S.f(F_CA)[i] = o.ca;
    S.f(F_R)[i] = o.r;
    S.f(F_S)[i] = o.s;
    S.f(F_Q)[i] = o.q;
    S.f(F_K)[i] = o.k;
    S.f(F_L)[i] = o.l;
    S.f(F_MS)[i] = o.ms;
    S.f(F_HS)[i] = o.hs;
    S.f(F_NS)[i] = o.ns;
    S.f(F_XS)[i] = o.xs;
    S.f(F_MA)[i] = o.ma;
    S.f(F_HA)[i] = o.ha;
    S.f(F_XA)[i] = o.xa;
    S.f(F_ICAH)[i] = o.icah;
    S.f(F_IC)[i] = o.ic;
}

// non-finite guard: a NaN or Inf in a voltage or [Ca] sets bit 0 of the status word
__device__ __forceinline__ bool cell_finite(const CellNext &o) {
    return isfinite(o.vd) && isfinite(o.vs) && isfinite(o.va) && isfinite(o.ca);
}

// ---- evoked input -----------------------------------------------------------------
// Pulse table grouped by cell: the pulses of cell i are [off[i], off[i+1]).
struct PulseTable {
    const int32_t *off;     // n + 1 (NULL: no pulses)
    const int64_t *begin;
    const int64_t *end;
    const float *amp;
};
__device__ __forceinline__ float pulse_current_range(const PulseTable &T, int32_t p0, int32_t p1, int64_t t) {
    float I = 0.0f;
    for (int32_t p = p0; p < p1; ++p)
        if (t >= T.begin[p] && t < T.end[p]) I += T.amp[p];
    return I;
}
__device__ __forceinline__ float pulse_current(const PulseTable &T, int64_t i, int64_t t) {
    if (T.off == nullptr) return 0.0f;
    return pulse_current_range(T, T.off[i], T.off[i + 1], t);
}

// Status word bits set by kernels (sticky until read by the host).
enum StatusBits : uint32_t { ST_NONFINITE = 1u, ST_TIMEOUT = 2u, ST_SLOT = 4u };

}  // namespace ion
