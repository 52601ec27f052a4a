// lowering.cu -- circuit gates to the planners' gate form.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace qsim {

bool commute(const SGate &a, const SGate &b)
{
    const uint64_t shared = (a.xq() | a.dq()) & (b.xq() | b.dq());
    return (shared & (a.xq() | b.xq())) == 0;
}

// SWAP(a, b) with controls c = CNOT(b -> a) . X(target b; controls c + a) . CNOT(b -> a)
void lower_gates(const sim_gate *gates, size_t n_gates, std::vector<SGate> *out)
{
    static const double X[8] = {0, 0, 1, 0, 1, 0, 0, 0};
    for (size_t k = 0; k < n_gates; ++k) {
        const PairGate p = make_pair_gate(gates[k]);
        uint64_t cm = 0;
        for (int c = 0; c < p.nctrl; ++c) cm |= 1ull << p.ctrl[c];
        if (p.op == OP_IDENTITY) continue;
        if (p.op == OP_SWAP) {
            const int a = p.target, b = p.target2;
            SGate g1{OP_XPERM, a, 1ull << b, {}, (int)k};
            SGate g2{OP_XPERM, b, cm | (1ull << a), {}, (int)k};
            memcpy(g1.m, X, sizeof X);
            memcpy(g2.m, X, sizeof X);
            out->push_back(g1);
            out->push_back(g2);
            out->push_back(g1);
            continue;
        }
        SGate g{p.op, p.target, cm, {}, (int)k};
        memcpy(g.m, p.m, sizeof g.m);
        out->push_back(g);
    }
}

double sgate_flops(const SGate &g, int n)
{
    const double amps = std::ldexp(1.0, n - __builtin_popcountll(g.ctrl));
    switch (g.op) {
    case OP_DENSE: return 16.0 * amps;                 // two complex MACs per amplitude
    case OP_ANTIDIAG: return 6.0 * amps;               // one complex multiply per amplitude
    case OP_DIAG: return 6.0 * amps;
    case OP_DIAG_HI:                                   // only the |1> half; a sign flip is a move
        return (g.m[6] == -1.0 && g.m[7] == 0.0) ? 0.0 : 3.0 * amps;
    case OP_SUPER: return 32.0 * amps;                 // four complex MACs per amplitude
    default: return 0.0;                               // exchanges
    }
}

}  // namespace qsim
