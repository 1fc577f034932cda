// flop_count.cpp -- operation counts of the oracle's cell step and gap-junction term,
// taken with an instrumented number type (TEST INFRASTRUCTURE ONLY; built and run by the
// tests, never by the library).
//
// The paper quotes the work of one neuron as 859 floating-point operations per step and
// one gap junction as 12 (Sec. 2.2, Table "reqs"), without saying how an exponential or
// a division is counted.  This program compiles the unchanged oracle source with every
// `double` replaced by a number type that counts each addition/subtraction,
// multiplication, division, exponential (exp, expm1), min/max and comparison, runs one
// cell step, one dense 2-cell gap-junction pass and one SGJ pass (Sec. 2.3.2 quotes 4
// operations per connection), and prints the counts as
// `name value` lines.  A sign change is not counted.
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

namespace {
struct Counts {
    long add, mul, div, exp, minmax, cmp;
};
Counts g_count;
}  // namespace

struct Flop {
    double v;
    Flop() = default;
    Flop(double x) : v(x) {}   // literals and the oracle's float inputs convert implicitly
    explicit operator double() const { return v; }
};
inline Flop operator+(Flop a, Flop b) { ++g_count.add; return Flop(a.v + b.v); }
inline Flop operator-(Flop a, Flop b) { ++g_count.add; return Flop(a.v - b.v); }
inline Flop operator*(Flop a, Flop b) { ++g_count.mul; return Flop(a.v * b.v); }
inline Flop operator/(Flop a, Flop b) { ++g_count.div; return Flop(a.v / b.v); }
inline Flop operator-(Flop a) { return Flop(-a.v); }
inline Flop &operator+=(Flop &a, Flop b) { a = a + b; return a; }
inline Flop &operator-=(Flop &a, Flop b) { a = a - b; return a; }
inline Flop &operator*=(Flop &a, Flop b) { a = a * b; return a; }
inline Flop &operator/=(Flop &a, Flop b) { a = a / b; return a; }
inline bool operator==(Flop a, Flop b) { ++g_count.cmp; return a.v == b.v; }
inline bool operator!=(Flop a, Flop b) { ++g_count.cmp; return a.v != b.v; }
inline bool operator<(Flop a, Flop b) { ++g_count.cmp; return a.v < b.v; }
inline bool operator>(Flop a, Flop b) { ++g_count.cmp; return a.v > b.v; }
inline bool operator<=(Flop a, Flop b) { ++g_count.cmp; return a.v <= b.v; }
inline bool operator>=(Flop a, Flop b) { ++g_count.cmp; return a.v >= b.v; }
inline Flop exp(Flop a) { ++g_count.exp; return Flop(std::exp(a.v)); }
inline Flop expm1(Flop a) { ++g_count.exp; return Flop(std::expm1(a.v)); }
inline Flop fmin(Flop a, Flop b) { ++g_count.minmax; return Flop(std::fmin(a.v, b.v)); }
inline Flop fmax(Flop a, Flop b) { ++g_count.minmax; return Flop(std::fmax(a.v, b.v)); }

#define double Flop
#include "ion_oracle.c"
#undef double

static void report(const char *what, const Counts &c, double per) {
    std::printf("%s_add %.3f\n%s_mul %.3f\n%s_div %.3f\n%s_exp %.3f\n%s_minmax %.3f\n%s_cmp %.3f\n", what,
                c.add / per, what, c.mul / per, what, c.div / per, what, c.exp / per, what, c.minmax / per, what,
                c.cmp / per);
}

int main() {
    Flop P[OP_NPARAMS];
    or_model_default(P);
    Flop S[OF_NFIELDS], Sn[OF_NFIELDS];
    or_default_state(1, P, S);
    S[OF_VDEND] = Flop(-55.0);   // away from rest, so no branch is at its special point
    Flop ic(0.25), iapp(1.0);
    g_count = Counts{};
    or_cell_step(1, P, nullptr, Flop(0.05), S, &ic, &iapp, Sn, 1);
    report("cell", g_count, 1.0);
    // one dense pass over 2 cells evaluates 4 ordered pairs (the self pairs included),
    // plus one multiplication by g per row
    Flop vd[2] = {Flop(-60.0), Flop(-52.5)}, icg[2];
    g_count = Counts{};
    or_gj_dense(2, vd, Flop(0.04), icg, 1);
    g_count.mul -= 2;
    report("gj_pair", g_count, 4.0);
    // the SGJ use case on the 2-cell CSR complete graph: one stored connection per row
    const int32_t rp[3] = {0, 1, 2}, col[2] = {1, 0};
    Flop w[2] = {Flop(0.04), Flop(0.04)};
    g_count = Counts{};
    or_gj_csr_sgj(2, rp, col, w, vd, icg, 1);
    report("sgj_edge", g_count, 2.0);
    return 0;
}
