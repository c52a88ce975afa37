/*
 * op_count.cpp -- counts the floating-point operations of one oracle time
 * step per lattice node (TEST INFRASTRUCTURE, like the rest of oracle/).
 *
 * lbm_oracle.c is compiled unchanged as C++ with every `double` replaced by
 * `tdouble`, a value that also records how it was computed.  Each arithmetic
 * operation of the oracle then becomes a node of an expression graph with
 * its FP64 value alongside (control flow follows the values, so the traced
 * step takes the oracle's own branches).  A node is counted as one
 * floating-point operation (add, subtract, multiply, divide or square root)
 * unless
 *   - all of its operands are constants: literals of the code or model
 *     parameters (A, kappa, G, s, the EOS constants), which a run fixes once;
 *   - it is an identity of a literal: x*1, x*(-1), x*0, x+0, x-0, 0-x, x/1,
 *     x/(-1), x-x (the integer entries of M and of the velocities make many);
 *     a negation is free (it folds into the consumer), and signs are taken
 *     out of products and quotients ((-c) x = -(c x) exactly), so that
 *     6 v.F and -6 v.F are one multiplication;
 *   - the same operation on the same operands was already counted (common
 *     subexpressions, e.g. psi^2 of a node used by all its neighbours, are
 *     counted once; + and * are commutative).
 * Model parameters are never treated as identities, even where a run sets one
 * to 1 or -1 (K = 1, G = -1): the count does not depend on their values.
 *
 * Output (stdout, one line per quantity): the counted operations of one time
 * step of an nx x ny periodic lattice divided by nx*ny, in total and by kind.
 * Usage: op_count <eos 1|2|3> <nx> <ny>   (kappa, A, s as in the spinodal
 * workload; the count does not depend on the field's values), or
 * op_count meq | source_s for the count of one of those two pieces alone.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <unordered_map>
#include <vector>

namespace opc {

enum Kind { LIT = 0, PARAM, VAR, ADD, SUB, MUL, DIV, SQRT, NEG, NKIND };

struct Node {
    int kind, a, b;
    double v;
};

std::vector<Node>& nodes() {
    static std::vector<Node> n{{LIT, -1, -1, 0.0}};   // node 0: the literal 0
    return n;
}
std::unordered_map<uint64_t, int>& table() {
    static std::unordered_map<uint64_t, int> t;
    return t;
}
long long g_count[NKIND] = {};

inline bool is_const(int id) { return nodes()[id].kind == LIT || nodes()[id].kind == PARAM; }
inline bool is_lit(int id, double v) { return nodes()[id].kind == LIT && nodes()[id].v == v; }

int make(int kind, int a, int b, double v) {
    nodes().push_back(Node{kind, a, b, v});
    return static_cast<int>(nodes().size()) - 1;
}

// constants are interned by kind and value, so equal ones are one node
int constant(double v, bool param) {
    static std::unordered_map<uint64_t, int> seen[2];
    if (v == 0.0 && !param) return 0;
    uint64_t bits;
    memcpy(&bits, &v, sizeof bits);
    auto it = seen[param].find(bits);
    if (it != seen[param].end()) return it->second;
    const int id = make(param ? PARAM : LIT, -1, -1, v);
    seen[param][bits] = id;
    return id;
}

// a counted operation, shared when the same one exists
int op(int kind, int a, int b, double v) {
    if ((kind == ADD || kind == MUL) && b >= 0 && a > b) { const int t = a; a = b; b = t; }
    const uint64_t key = (static_cast<uint64_t>(kind) << 58) ^ (static_cast<uint64_t>(static_cast<uint32_t>(a)) << 29) ^
                         static_cast<uint64_t>(static_cast<uint32_t>(b + 1));
    auto it = table().find(key);
    if (it != table().end()) {
        const Node& n = nodes()[it->second];
        if (n.kind == kind && ((n.a == a && n.b == b))) return it->second;
    }
    const int id = make(kind, a, b, v);
    table()[key] = id;
    ++g_count[kind];
    return id;
}

int neg(int a) {
    static std::unordered_map<int, int> seen;
    const Node n = nodes()[a];
    if (is_const(a)) return constant(-n.v, n.kind == PARAM);
    if (n.kind == NEG) return n.a;
    auto it = seen.find(a);
    if (it != seen.end()) return it->second;
    const int id = make(NEG, a, -1, -n.v);
    seen[a] = id;
    return id;
}

int param_or_lit(int a, int b) { return (nodes()[a].kind == PARAM || nodes()[b].kind == PARAM); }

int add(int a, int b);
int sub(int a, int b) {
    const double v = nodes()[a].v - nodes()[b].v;
    if (is_const(a) && is_const(b)) return constant(v, param_or_lit(a, b));
    if (a == b) return 0;
    if (is_lit(b, 0.0)) return a;
    if (is_lit(a, 0.0)) return neg(b);
    if (nodes()[b].kind == NEG) return add(a, nodes()[b].a);
    if (nodes()[a].kind == NEG) return neg(add(nodes()[a].a, b));
    return op(SUB, a, b, v);
}
int add(int a, int b) {
    const double v = nodes()[a].v + nodes()[b].v;
    if (is_const(a) && is_const(b)) return constant(v, param_or_lit(a, b));
    if (is_lit(b, 0.0)) return a;
    if (is_lit(a, 0.0)) return b;
    if (nodes()[b].kind == NEG) return sub(a, nodes()[b].a);
    if (nodes()[a].kind == NEG) return sub(b, nodes()[a].a);
    return op(ADD, a, b, v);
}
int mul(int a, int b) {
    const double v = nodes()[a].v * nodes()[b].v;
    if (is_const(a) && is_const(b)) return constant(v, param_or_lit(a, b));
    if (is_lit(a, 0.0) || is_lit(b, 0.0)) return 0;
    if (is_lit(b, 1.0)) return a;
    if (is_lit(a, 1.0)) return b;
    if (is_lit(b, -1.0)) return neg(a);
    if (is_lit(a, -1.0)) return neg(b);
    if (nodes()[a].kind == NEG) return neg(mul(nodes()[a].a, b));
    if (nodes()[b].kind == NEG) return neg(mul(a, nodes()[b].a));
    if (is_const(a) && nodes()[a].v < 0) return neg(mul(neg(a), b));   // (-c) x = -(c x) exactly
    if (is_const(b) && nodes()[b].v < 0) return neg(mul(a, neg(b)));
    return op(MUL, a, b, v);
}
int div(int a, int b) {
    const double v = nodes()[a].v / nodes()[b].v;
    if (is_const(a) && is_const(b)) return constant(v, param_or_lit(a, b));
    if (is_lit(a, 0.0)) return 0;
    if (is_lit(b, 1.0)) return a;
    if (is_lit(b, -1.0)) return neg(a);
    if (nodes()[a].kind == NEG) return neg(div(nodes()[a].a, b));
    if (nodes()[b].kind == NEG) return neg(div(a, nodes()[b].a));
    if (is_const(a) && nodes()[a].v < 0) return neg(div(neg(a), b));
    if (is_const(b) && nodes()[b].v < 0) return neg(div(a, neg(b)));
    return op(DIV, a, b, v);
}
int sqrt_(int a) {
    const double v = std::sqrt(nodes()[a].v);
    if (is_const(a)) return constant(v, nodes()[a].kind == PARAM);
    return op(SQRT, a, -1, v);
}

}  // namespace opc

// The traced FP64 value.  Conversions from int and double make literals.
struct tdouble {
    int id;
    tdouble() : id(0) {}
    tdouble(double v) : id(opc::constant(v, false)) {}
    tdouble(int v) : tdouble(static_cast<double>(v)) {}
    tdouble(long v) : tdouble(static_cast<double>(v)) {}
    static tdouble of(int i) { tdouble t; t.id = i; return t; }
    double value() const { return opc::nodes()[id].v; }
};
inline tdouble param(double v) { return tdouble::of(opc::constant(v, true)); }
inline tdouble var(double v) { return tdouble::of(opc::make(opc::VAR, -1, -1, v)); }

inline tdouble operator+(tdouble a, tdouble b) { return tdouble::of(opc::add(a.id, b.id)); }
inline tdouble operator-(tdouble a, tdouble b) { return tdouble::of(opc::sub(a.id, b.id)); }
inline tdouble operator*(tdouble a, tdouble b) { return tdouble::of(opc::mul(a.id, b.id)); }
inline tdouble operator/(tdouble a, tdouble b) { return tdouble::of(opc::div(a.id, b.id)); }
inline tdouble operator-(tdouble a) { return tdouble::of(opc::neg(a.id)); }
inline tdouble& operator+=(tdouble& a, tdouble b) { return a = a + b; }
inline tdouble& operator-=(tdouble& a, tdouble b) { return a = a - b; }
inline tdouble& operator*=(tdouble& a, tdouble b) { return a = a * b; }
inline bool operator<(tdouble a, tdouble b) { return a.value() < b.value(); }
inline bool operator>(tdouble a, tdouble b) { return a.value() > b.value(); }
inline bool operator<=(tdouble a, tdouble b) { return a.value() <= b.value(); }
inline bool operator>=(tdouble a, tdouble b) { return a.value() >= b.value(); }
inline bool operator==(tdouble a, tdouble b) { return a.value() == b.value(); }
inline bool operator!=(tdouble a, tdouble b) { return a.value() != b.value(); }
inline tdouble sqrt(tdouble a) { return tdouble::of(opc::sqrt_(a.id)); }

// the oracle itself, every double traced
#define double tdouble
#include "lbm_oracle.c"
#undef double

// Counts of two single-node pieces of the oracle with hand-countable
// arithmetic, so that the counting rules can be checked: the equilibrium
// moments of Eq. 4 and the forcing moments of Eq. 6.
static long long piece(const char* which) {
    long long c0[opc::NKIND];
    memcpy(c0, opc::g_count, sizeof c0);
    tdouble out[9];
    if (strcmp(which, "meq") == 0) orc_meq(var(0.3), var(0.01), var(-0.02), out);
    else orc_source_s(var(0.01), var(-0.02), var(1e-4), var(2e-4), out);
    long long n = 0;
    for (int k = opc::ADD; k <= opc::SQRT; ++k) n += opc::g_count[k] - c0[k];
    return n;
}

int main(int argc, char** argv) {
    if (argc == 2 && (strcmp(argv[1], "meq") == 0 || strcmp(argv[1], "source_s") == 0)) {
        printf("flops=%lld\n", piece(argv[1]));
        return 0;
    }
    if (argc < 4) {
        fprintf(stderr, "usage: %s <eos 1|2|3> <nx> <ny> | meq | source_s\n", argv[0]);
        return 2;
    }
    const int eos = atoi(argv[1]), nx = atoi(argv[2]), ny = atoi(argv[3]);
    if (eos < 1 || eos > 3 || nx < 3 || ny < 3) return 2;
    orc_params p;
    memset(static_cast<void*>(&p), 0, sizeof p);
    p.eos = eos;
    // constants of the workloads of each law (their values do not change the count)
    const double a = eos == 1 ? 1.0 : (eos == 2 ? 9.0 / 49.0 : 0.0703), b = eos == 1 ? 4.0 : 2.0 / 21.0;
    const double T = eos == 1 ? 0.066 : (eos == 2 ? 0.3 : 0.09);
    p.a = param(a);
    p.b = param(b);
    p.R = param(1.0);
    p.K = param(eos == 2 ? 0.3 : 1.0);
    p.T = param(T);
    p.omega = param(0.344);
    p.Tc = param(eos == 3 ? 0.1136 : 0.0);
    p.A = param(-0.85);
    p.kappa = param(0.3);
    p.G = param(-1.0);
    const double s[9] = {1.0, 1.1, 1.1, 1.0, 1.1, 1.0, 1.1, 1.0, 1.0};
    for (int k = 0; k < 9; ++k) p.s[k] = param(s[k]);
    p.fext_x = param(0.0);
    p.fext_y = param(0.0);
    p.nu_g = p.nu_l = p.visc_rho_g = p.visc_rho_l = param(0.0);

    // a field inside the law's psi domain: populations of rho ~ 0.2 b^-1 ... with
    // small seeded variations, so that no two nodes hold equal values
    const long N = static_cast<long>(nx) * ny;
    std::vector<tdouble> f(9 * N);
    unsigned long long z = 14127228ull;
    const double t[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    const double rho0 = (eos == 1 ? 0.25 : 1.5 * (eos == 2 ? 1.0 : 0.5));
    for (long i = 0; i < N; ++i)
        for (int q = 0; q < 9; ++q) {
            z = z * 6364136223846793005ull + 1442695040888963407ull;
            const double u = static_cast<double>(z >> 11) / 9007199254740992.0;
            f[q * N + i] = var(t[q] * rho0 * (1.0 + 0.01 * (2.0 * u - 1.0)));
        }
    long long c0[opc::NKIND];
    memcpy(c0, opc::g_count, sizeof c0);
    const int rc = orc_step(&p, nx, ny, f.data(), 1);
    if (rc != 0) {
        fprintf(stderr, "oracle step failed: %d\n", rc);
        return 1;
    }
    long long d[opc::NKIND];
    for (int k = 0; k < opc::NKIND; ++k) d[k] = opc::g_count[k] - c0[k];
    const double n = static_cast<double>(N);
    const long long total = d[opc::ADD] + d[opc::SUB] + d[opc::MUL] + d[opc::DIV] + d[opc::SQRT];
    printf("flops_per_update=%.6f\n", total / n);
    printf("add_sub_per_update=%.6f\n", (d[opc::ADD] + d[opc::SUB]) / n);
    printf("mul_per_update=%.6f\n", d[opc::MUL] / n);
    printf("div_per_update=%.6f\n", d[opc::DIV] / n);
    printf("sqrt_per_update=%.6f\n", d[opc::SQRT] / n);
    return 0;
}
