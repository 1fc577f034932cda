/*
 * ion_oracle.c -- plain FP64 CPU oracle of the InfOli inferior-olive network step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg do.  It
 * shares no code, header, table or helper with the CUDA path: its constants table is
 * its own copy, and the tests compare the two copies.
 *
 * What it computes (paper: Smaragdos et al., "BrainFrame", arXiv 1612.01501):
 *   - Sec. 2.2 ("The InfOli Workload"): every new neuron state depends only on the
 *     cell's own previous state, the previous dendritic voltages of the cells it is
 *     gap-junction coupled to, and the evoked input.  The three compartments and the
 *     gap junctions are updated concurrently, with a fixed step delta = 50 us.  We read
 *     "concurrently" as pure explicit (forward) Euler: every right-hand side is
 *     evaluated from step-t values only, and the step-(t+1) state is written elsewhere.
 *   - Algorithm 1 (RGJ): for each connection, V = V_dend,i - V_dend,j and the cell
 *     accumulates Ic += w * (0.8 * exp(-V*V/100) + 0.2) * V.  The printed listing has
 *     an extra factor V inside f; we take the odd form (0.8 e^{-V^2/100} + 0.2) V,
 *     which keeps I_ij = -I_ji (the antisymmetry the tests check).
 *   - Sec. 2.3 / Table "reqs": the connectivity is a user-programmable N x N matrix of
 *     weights; a dense uniform all-to-all network uses one weight g_c for every pair
 *     (the j = i term is exactly zero and is summed like any other).
 *   - Sec. 2.2 (the model is De Gruijl et al. 2012's three-compartment cell): the cell
 *     equations are not printed in the paper.  The ones below are the published
 *     three-compartment IO cell (dendrite: high-threshold Ca, Ca-activated K, h-current,
 *     leak, [Ca] pool; soma: low-threshold Ca, Na, delayed-rectifier K, voltage-gated K,
 *     leak; axon: Na, K, leak; ohmic dendrite-soma and soma-axon coupling), written from
 *     the model's equations.  Parity of these constants with the publication is
 *     unpinned (the publication is not available here); parity between this oracle and
 *     the GPU path is pinned because both consume tables with the same values.
 *
 * Units: mV, ms, mS/cm^2, uF/cm^2, uA/cm^2; [Ca] in the model's arbitrary units.
 * Layout: state is structure-of-arrays, S[f * n + i] for field f of cell i, with the
 * 19 fields below (Table "reqs" gives 19 state words per neuron).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- state fields (19 words per cell, Table "reqs") ---------------------------- */
enum {
    OF_VDEND = 0, /* dendritic membrane voltage                                       */
    OF_VSOMA,     /* somatic membrane voltage                                         */
    OF_VAXON,     /* axonal membrane voltage (the cell output)                         */
    OF_CA,        /* dendritic calcium concentration                                   */
    OF_R,         /* high-threshold Ca activation (dendrite)                           */
    OF_S,         /* Ca-activated K activation (dendrite, [Ca]-gated)                  */
    OF_Q,         /* h-current activation (dendrite)                                   */
    OF_K,         /* low-threshold Ca activation (soma)                                */
    OF_L,         /* low-threshold Ca inactivation (soma)                              */
    OF_MS,        /* Na activation (soma), instantaneous: holds m_inf(V_soma) of step t */
    OF_HS,        /* Na inactivation (soma)                                            */
    OF_NS,        /* delayed-rectifier K activation (soma)                             */
    OF_XS,        /* voltage-gated K activation (soma)                                 */
    OF_MA,        /* Na activation (axon), instantaneous: holds m_inf(V_axon) of step t */
    OF_HA,        /* Na inactivation (axon)                                            */
    OF_XA,        /* voltage-gated K activation (axon)                                 */
    OF_GCAL,      /* per-cell low-threshold Ca conductance (constant in time)          */
    OF_ICAH,      /* high-threshold Ca current used in step t (drives the [Ca] pool)   */
    OF_IC,        /* gap-junction current used in step t                               */
    OF_NFIELDS
};

/* ---- constants table (this oracle's own copy) ----------------------------------- */
enum {
    OP_GINT = 0, OP_P1, OP_P2,                           /* coupling                    */
    OP_GCAH, OP_GKCA, OP_GH, OP_GLD,                     /* dendrite conductances       */
    OP_GCAL, OP_GNAS, OP_GKDRS, OP_GKS, OP_GLS,          /* soma conductances           */
    OP_GNAA, OP_GKA, OP_GLA,                             /* axon conductances           */
    OP_VNA, OP_VK, OP_VCA, OP_VH, OP_VL,                 /* reversal potentials         */
    OP_CM,                                               /* membrane capacitance        */
    OP_CA_IN, OP_CA_OUT,                                 /* [Ca] influx / decay factors */
    OP_V0, OP_CA0,                                       /* default initial state       */
    OP_NPARAMS
};

static const double or_default_table[OP_NPARAMS] = {
    /* g_int  */ 0.13,  /* p1 (soma share of the dendrite-soma pair) */ 0.25,
    /* p2 (axon share of the soma-axon pair) */ 0.15,
    /* g_CaH  */ 4.5,   /* g_KCa  */ 35.0,  /* g_h    */ 0.125, /* g_ld   */ 0.016,
    /* g_CaL  */ 0.68,  /* g_Na_s */ 150.0, /* g_Kdr_s*/ 9.0,   /* g_K_s  */ 5.0,
    /* g_ls   */ 0.016,
    /* g_Na_a */ 240.0, /* g_K_a  */ 20.0,  /* g_la   */ 0.016,
    /* V_Na   */ 55.0,  /* V_K    */ -75.0, /* V_Ca   */ 120.0, /* V_h    */ -43.0,
    /* V_L    */ 10.0,
    /* C_m    */ 1.0,
    /* [Ca] influx per unit I_CaH */ 3.0, /* [Ca] decay rate (1/ms) */ 0.075,
    /* V_0    */ -60.0, /* [Ca]_0 */ 3.715,
};

int or_nfields(void) { return OF_NFIELDS; }
int or_nparams(void) { return OP_NPARAMS; }

void or_model_default(double *out) { memcpy(out, or_default_table, sizeof or_default_table); }

/* ---- channel kinetics ------------------------------------------------------------
 * Each gate x relaxes as dx/dt = (x_inf(V) - x) / tau_x(V).  Gate order (12 gates):
 *   0 r, 1 s, 2 q (dendrite; s is a function of [Ca] only),
 *   3 k, 4 l, 5 m_s, 6 h_s, 7 n_s, 8 x_s (soma),
 *   9 m_a, 10 h_a, 11 x_a (axon).
 * m_s and m_a are instantaneous (tau reported as 0).
 */
enum { OG_R, OG_S, OG_Q, OG_K, OG_L, OG_MS, OG_HS, OG_NS, OG_XS, OG_MA, OG_HA, OG_XA, OG_NGATES };
int or_ngates(void) { return OG_NGATES; }

static double sigmoid_rise(double V, double vhalf, double slope) { /* 1/(1+e^{-(V-vh)/k}) */
    return 1.0 / (1.0 + exp(-(V - vhalf) / slope));
}
static double sigmoid_fall(double V, double vhalf, double slope) { /* 1/(1+e^{(V-vh)/k}) */
    return 1.0 / (1.0 + exp((V - vhalf) / slope));
}
/* z / (e^z - 1), continuous at z = 0 where it equals 1 */
static double z_over_expm1(double z) { return z == 0.0 ? 1.0 : z / expm1(z); }

/* high-threshold Ca (dendrite): alpha, beta in 1/ms */
static void rate_r(double V, double *xinf, double *tau) {
    double a = 1.7 / (1.0 + exp(-(V - 5.0) / 13.9));
    double b = 0.02 * 5.0 * z_over_expm1((V + 8.5) / 5.0); /* 0.02 (V+8.5)/(e^{(V+8.5)/5}-1) */
    *xinf = a / (a + b);
    *tau = 5.0 / (a + b);
}
/* Ca-activated K (dendrite): alpha = min(2e-5 [Ca], 0.01), beta = 0.015 */
static void rate_s(double ca, double *xinf, double *tau) {
    double a = fmin(2.0e-5 * ca, 0.01);
    double b = 0.015;
    *xinf = a / (a + b);
    *tau = 1.0 / (a + b);
}
/* h-current (dendrite) */
static void rate_q(double V, double *xinf, double *tau) {
    *xinf = sigmoid_fall(V, -80.0, 4.0);
    *tau = 1.0 / (exp(-0.086 * V - 14.6) + exp(0.070 * V - 1.87));
}
/* low-threshold Ca activation (soma) */
static void rate_k(double V, double *xinf, double *tau) {
    *xinf = sigmoid_rise(V, -61.0, 4.2);
    *tau = 1.0;
}
/* low-threshold Ca inactivation (soma) */
static void rate_l(double V, double *xinf, double *tau) {
    *xinf = sigmoid_fall(V, -85.5, 8.5);
    *tau = 20.0 * exp((V + 160.0) / 30.0) / (1.0 + exp((V + 84.0) / 7.3)) + 35.0;
}
/* Na activation (soma and axon), instantaneous */
static double minf_na(double V) { return sigmoid_rise(V, -30.0, 5.5); }
/* Na inactivation (soma) */
static void rate_hs(double V, double *xinf, double *tau) {
    *xinf = sigmoid_fall(V, -70.0, 5.8);
    *tau = 3.0 * exp(-(V + 40.0) / 33.0);
}
/* delayed-rectifier K (soma) */
static void rate_ns(double V, double *xinf, double *tau) {
    *xinf = sigmoid_rise(V, -3.0, 10.0);
    *tau = 5.0 + 47.0 * exp((V + 50.0) / 900.0);
}
/* voltage-gated K (soma and axon): alpha = 0.13 (V+25)/(1-e^{-(V+25)/10}),
 * beta = 1.69 e^{-0.0125 (V+35)} */
static void rate_x(double V, double *xinf, double *tau) {
    double y = (V + 25.0) / 10.0;
    double a = 0.13 * 10.0 * z_over_expm1(-y); /* y/(1-e^{-y}) = (-y)/(e^{-y}-1) */
    double b = 1.69 * exp(-0.0125 * (V + 35.0));
    *xinf = a / (a + b);
    *tau = 1.0 / (a + b);
}
/* Na inactivation (axon) */
static void rate_ha(double V, double *xinf, double *tau) {
    *xinf = sigmoid_fall(V, -60.0, 5.8);
    *tau = 1.5 * exp(-(V + 40.0) / 33.0);
}

/* All 12 gates evaluated at one voltage V and one [Ca]; x_inf and tau each hold 12. */
void or_rates(double V, double ca, double *xinf, double *tau) {
    rate_r(V, &xinf[OG_R], &tau[OG_R]);
    rate_s(ca, &xinf[OG_S], &tau[OG_S]);
    rate_q(V, &xinf[OG_Q], &tau[OG_Q]);
    rate_k(V, &xinf[OG_K], &tau[OG_K]);
    rate_l(V, &xinf[OG_L], &tau[OG_L]);
    xinf[OG_MS] = minf_na(V); tau[OG_MS] = 0.0;
    rate_hs(V, &xinf[OG_HS], &tau[OG_HS]);
    rate_ns(V, &xinf[OG_NS], &tau[OG_NS]);
    rate_x(V, &xinf[OG_XS], &tau[OG_XS]);
    xinf[OG_MA] = minf_na(V); tau[OG_MA] = 0.0;
    rate_ha(V, &xinf[OG_HA], &tau[OG_HA]);
    rate_x(V, &xinf[OG_XA], &tau[OG_XA]);
}

/* ---- default initial state -------------------------------------------------------
 * The paper gives no initial state.  Reading: every compartment at V_0, each gate at
 * its steady state x_inf(V_0) of its own compartment, [Ca] at [Ca]_0, s at s_inf([Ca]_0),
 * g_CaL at the table value, I_CaH the current of that state, I_c = 0.
 */
void or_default_state(int n, const double *P, double *S) {
    double V0 = P[OP_V0], ca0 = P[OP_CA0];
    double xi[OG_NGATES], ta[OG_NGATES];
    or_rates(V0, ca0, xi, ta);
    for (int i = 0; i < n; ++i) {
        S[OF_VDEND * n + i] = V0;
        S[OF_VSOMA * n + i] = V0;
        S[OF_VAXON * n + i] = V0;
        S[OF_CA * n + i] = ca0;
        S[OF_R * n + i] = xi[OG_R];
        S[OF_S * n + i] = xi[OG_S];
        S[OF_Q * n + i] = xi[OG_Q];
        S[OF_K * n + i] = xi[OG_K];
        S[OF_L * n + i] = xi[OG_L];
        S[OF_MS * n + i] = xi[OG_MS];
        S[OF_HS * n + i] = xi[OG_HS];
        S[OF_NS * n + i] = xi[OG_NS];
        S[OF_XS * n + i] = xi[OG_XS];
        S[OF_MA * n + i] = xi[OG_MA];
        S[OF_HA * n + i] = xi[OG_HA];
        S[OF_XA * n + i] = xi[OG_XA];
        S[OF_GCAL * n + i] = P[OP_GCAL];
        S[OF_ICAH * n + i] = P[OP_GCAH] * xi[OG_R] * xi[OG_R] * (V0 - P[OP_VCA]);
        S[OF_IC * n + i] = 0.0;
    }
}

/* ---- gap junctions (Algorithm 1) ------------------------------------------------ */

/* one connection's contribution, weight excluded: (0.8 e^{-dV^2/100} + 0.2) dV */
static double gj_term(double dv) { return (0.8 * exp(-dv * dv / 100.0) + 0.2) * dv; }

/* dense uniform all-to-all: Ic_i = g * sum_{j=0}^{n-1} term(V_i - V_j), j ascending */
void or_gj_dense(int n, const double *vd, double g, double *ic, int threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += gj_term(vd[i] - vd[j]);
        ic[i] = g * acc;
    }
    (void)threads;
}

/* CSR: Ic_i = sum_{e in row i} w_e * term(V_i - V_{col_e}), edges in stored order */
void or_gj_csr(int n, const int32_t *row_ptr, const int32_t *col, const double *w,
               const double *vd, double *ic, int threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) acc += w[e] * gj_term(vd[i] - vd[col[e]]);
        ic[i] = acc;
    }
    (void)threads;
}

/* dense N x N weight matrix (row-major, the programmed connectivity of Sec. 2.3 with every
 * pair stored): Ic_i = sum_{j=0}^{n-1} W[i][j] * term(V_i - V_j), j ascending */
void or_gj_matrix(int n, const double *W, const double *vd, double *ic, int threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += W[(size_t)i * (size_t)n + (size_t)j] * gj_term(vd[i] - vd[j]);
        ic[i] = acc;
    }
    (void)threads;
}

/* ---- simplified gap junctions (SGJ use case, Sec. 2.3.2) -------------------------
 * The paper replaces the junction kinetics by simple weighted accumulators (4 operations
 * per connection).  Read as a linear junction: each connection contributes w (V_i - V_j),
 * the small-dV limit of the RGJ term (0.8 + 0.2 = 1). */

/* dense uniform all-to-all: Ic_i = g * sum_{j=0}^{n-1} (V_i - V_j), j ascending */
void or_gj_dense_sgj(int n, const double *vd, double g, double *ic, int threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int j = 0; j < n; ++j) acc += vd[i] - vd[j];
        ic[i] = g * acc;
    }
    (void)threads;
}

/* CSR: Ic_i = sum_{e in row i} w_e * (V_i - V_{col_e}), edges in stored order */
void or_gj_csr_sgj(int n, const int32_t *row_ptr, const int32_t *col, const double *w,
                   const double *vd, double *ic, int threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) acc += w[e] * (vd[i] - vd[col[e]]);
        ic[i] = acc;
    }
    (void)threads;
}

/* ---- cell update (explicit Euler, all right-hand sides from step t) -------------- */

/* Per-cell constants (Table "reqs": each neuron has its own conductances).  Pc, when not
 * NULL, holds OP_NCELL values per cell, structure of arrays (entry p of cell i at
 * Pc[p * n + i], p in table order 0..19); they replace the table's entries for that cell,
 * except g_CaL, which is per cell already (state field OF_GCAL). */
enum { OP_NCELL = 20 };

static void cell_step_one(int n, int i, const double *P_table, const double *Pc, double dt, const double *S,
                          double ic, double iapp, double *Sn) {
    double P_cell[OP_NPARAMS];
    const double *P = P_table;
    if (Pc) {
        memcpy(P_cell, P_table, sizeof P_cell);
        for (int p = 0; p < OP_NCELL; ++p)
            if (p != OP_GCAL) P_cell[p] = Pc[(size_t)p * (size_t)n + (size_t)i];
        P = P_cell;
    }
#define F(f) S[(f) * n + i]
    const double Vd = F(OF_VDEND), Vs = F(OF_VSOMA), Va = F(OF_VAXON), ca = F(OF_CA);
    const double Cm = P[OP_CM];
    double xi_d[OG_NGATES], ta_d[OG_NGATES];
    double xi_s[OG_NGATES], ta_s[OG_NGATES];
    double xi_a[OG_NGATES], ta_a[OG_NGATES];
    or_rates(Vd, ca, xi_d, ta_d); /* dendrite gates use V_dend (s uses [Ca]) */
    or_rates(Vs, ca, xi_s, ta_s); /* soma gates use V_soma */
    or_rates(Va, ca, xi_a, ta_a); /* axon gates use V_axon */

    /* dendrite currents */
    const double r = F(OF_R), s = F(OF_S), q = F(OF_Q);
    const double I_CaH = P[OP_GCAH] * r * r * (Vd - P[OP_VCA]);
    const double I_KCa = P[OP_GKCA] * s * (Vd - P[OP_VK]);
    const double I_h = P[OP_GH] * q * (Vd - P[OP_VH]);
    const double I_ld = P[OP_GLD] * (Vd - P[OP_VL]);
    const double I_ds = P[OP_GINT] / (1.0 - P[OP_P1]) * (Vd - Vs);
    const double dVd = (iapp - I_CaH - I_KCa - I_h - I_ld - I_ds - ic) / Cm;
    const double dCa = -P[OP_CA_IN] * I_CaH - P[OP_CA_OUT] * ca;

    /* soma currents */
    const double k = F(OF_K), l = F(OF_L), hs = F(OF_HS), ns = F(OF_NS), xs = F(OF_XS);
    const double ms = xi_s[OG_MS];
    const double I_CaL = F(OF_GCAL) * k * k * k * l * (Vs - P[OP_VCA]);
    const double I_Na_s = P[OP_GNAS] * ms * ms * ms * hs * (Vs - P[OP_VNA]);
    const double I_Kdr = P[OP_GKDRS] * ns * ns * ns * ns * (Vs - P[OP_VK]);
    const double I_K_s = P[OP_GKS] * xs * xs * xs * xs * (Vs - P[OP_VK]);
    const double I_ls = P[OP_GLS] * (Vs - P[OP_VL]);
    const double I_sd = P[OP_GINT] / P[OP_P1] * (Vs - Vd);
    const double I_sa = P[OP_GINT] / (1.0 - P[OP_P2]) * (Vs - Va);
    const double dVs = -(I_CaL + I_Na_s + I_Kdr + I_K_s + I_ls + I_sd + I_sa) / Cm;

    /* axon currents */
    const double ha = F(OF_HA), xa = F(OF_XA);
    const double ma = xi_a[OG_MA];
    const double I_Na_a = P[OP_GNAA] * ma * ma * ma * ha * (Va - P[OP_VNA]);
    const double I_K_a = P[OP_GKA] * xa * xa * xa * xa * (Va - P[OP_VK]);
    const double I_la = P[OP_GLA] * (Va - P[OP_VL]);
    const double I_as = P[OP_GINT] / P[OP_P2] * (Va - Vs);
    const double dVa = -(I_Na_a + I_K_a + I_la + I_as) / Cm;
#undef F
#define G(f) Sn[(f) * n + i]
    G(OF_VDEND) = Vd + dt * dVd;
    G(OF_VSOMA) = Vs + dt * dVs;
    G(OF_VAXON) = Va + dt * dVa;
    G(OF_CA) = ca + dt * dCa;
    G(OF_R) = r + dt * (xi_d[OG_R] - r) / ta_d[OG_R];
    G(OF_S) = s + dt * (xi_d[OG_S] - s) / ta_d[OG_S];
    G(OF_Q) = q + dt * (xi_d[OG_Q] - q) / ta_d[OG_Q];
    G(OF_K) = k + dt * (xi_s[OG_K] - k) / ta_s[OG_K];
    G(OF_L) = l + dt * (xi_s[OG_L] - l) / ta_s[OG_L];
    G(OF_MS) = ms;
    G(OF_HS) = hs + dt * (xi_s[OG_HS] - hs) / ta_s[OG_HS];
    G(OF_NS) = ns + dt * (xi_s[OG_NS] - ns) / ta_s[OG_NS];
    G(OF_XS) = xs + dt * (xi_s[OG_XS] - xs) / ta_s[OG_XS];
    G(OF_MA) = ma;
    G(OF_HA) = ha + dt * (xi_a[OG_HA] - ha) / ta_a[OG_HA];
    G(OF_XA) = xa + dt * (xi_a[OG_XA] - xa) / ta_a[OG_XA];
    G(OF_GCAL) = S[OF_GCAL * n + i];
    G(OF_ICAH) = I_CaH;
    G(OF_IC) = ic;
#undef G
}

/* Advance every cell one step: Sn = S + dt * F(S, ic, iapp).  S and Sn must not alias.
 * Pc: per-cell constants or NULL (see cell_step_one). */
void or_cell_step(int n, const double *P, const double *Pc, double dt, const double *S, const double *ic,
                  const double *iapp, double *Sn, int threads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : 1)
#endif
    for (int i = 0; i < n; ++i) cell_step_one(n, i, P, Pc, dt, S, ic ? ic[i] : 0.0, iapp ? iapp[i] : 0.0, Sn);
    (void)threads;
}

/* ---- whole run -------------------------------------------------------------------
 * kind 0: dense uniform all-to-all with weight g.  kind 1: CSR (row_ptr, col, w).
 * kind 2: no gap junctions (every cell independent).  kinds 3 and 4: as 0 and 1 with the
 * simplified (linear) junctions of the SGJ use case.  kind 5: dense N x N weight matrix
 * (w holds n * n row-major weights).
 * Evoked input at absolute step t (t0 <= t < t0 + n_steps), cell i:
 *   iapp_dense != NULL: iapp_dense[(t - t0) * n + i];
 *   else the sum of amp[p] over pulses p with cell[p] == i and t_begin[p] <= t < t_end[p].
 * S (19 * n, SoA) holds the step-t0 state on entry and the step-(t0 + n_steps) state on
 * return.  If trace != NULL, trace[(t - t0) * n_trace + c] = V_axon of cell
 * trace_cells[c] after step t.  Pc: per-cell constants or NULL (see cell_step_one).
 * Returns 0, or -1 if scratch could not be allocated.
 */
int or_run(int n, int kind, double g, const int32_t *row_ptr, const int32_t *col,
           const double *w, const double *P, const double *Pc, double dt, double *S, int64_t t0,
           int64_t n_steps, const float *iapp_dense, int n_pulses, const int32_t *p_cell,
           const int64_t *p_begin, const int64_t *p_end, const double *p_amp,
           int n_trace, const int32_t *trace_cells, double *trace, int threads) {
    double *Sn = malloc(sizeof(double) * (size_t)OF_NFIELDS * (size_t)n);
    double *ic = malloc(sizeof(double) * (size_t)n);
    double *vd = malloc(sizeof(double) * (size_t)n);
    double *iapp = malloc(sizeof(double) * (size_t)n);
    if (!Sn || !ic || !vd || !iapp) {
        free(Sn); free(ic); free(vd); free(iapp);
        return -1;
    }
    for (int64_t st = 0; st < n_steps; ++st) {
        const int64_t t = t0 + st;
        memcpy(vd, &S[OF_VDEND * n], sizeof(double) * (size_t)n);
        if (kind == 0) or_gj_dense(n, vd, g, ic, threads);
        else if (kind == 1) or_gj_csr(n, row_ptr, col, w, vd, ic, threads);
        else if (kind == 3) or_gj_dense_sgj(n, vd, g, ic, threads);
        else if (kind == 4) or_gj_csr_sgj(n, row_ptr, col, w, vd, ic, threads);
        else if (kind == 5) or_gj_matrix(n, w, vd, ic, threads);
        else memset(ic, 0, sizeof(double) * (size_t)n);
        if (iapp_dense) {
            for (int i = 0; i < n; ++i) iapp[i] = (double)iapp_dense[(size_t)st * (size_t)n + (size_t)i];
        } else {
            memset(iapp, 0, sizeof(double) * (size_t)n);
            for (int p = 0; p < n_pulses; ++p)
                if (t >= p_begin[p] && t < p_end[p]) iapp[p_cell[p]] += p_amp[p];
        }
        or_cell_step(n, P, Pc, dt, S, ic, iapp, Sn, threads);
        memcpy(S, Sn, sizeof(double) * (size_t)OF_NFIELDS * (size_t)n);
        if (trace)
            for (int c = 0; c < n_trace; ++c)
                trace[(size_t)st * (size_t)n_trace + (size_t)c] = S[OF_VAXON * n + trace_cells[c]];
    }
    free(Sn); free(ic); free(vd); free(iapp);
    return 0;
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
