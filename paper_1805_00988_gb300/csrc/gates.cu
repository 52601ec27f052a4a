// gates.cu -- per-gate kernels: one pass over the state per gate.
//
// Algorithm 1 (§2.3) updates every amplitude pair (a, b = a | 2^t) whose bit
// t of a is 0; the controlled form (§2.3, App. B.2) restricts it to pairs
// whose control bits are all 1.  Unlike the App. B.2 kernel, which visits all
// 2^(n-1) pairs and tests the control, these kernels enumerate only the pairs
// that change: the base index of work item w is w with zero bits inserted at
// the sorted positions {target, controls}, then the control bits set.  So a
// gate with c controls reads and writes 2S / 2^c bytes (S = state bytes), a
// phase gate on |1> only the half it multiplies, CNOT / Toffoli are pure moves.
//
// Memory access: complex64 work items carry two neighbouring amplitudes in one
// 16-byte vector (when no involved qubit is bit 0), complex128 items one
// 16-byte amplitude; each thread keeps U items in flight so the kernels are
// HBM-bound.  A target on bit 0 (complex64) loads the pair as one 16-byte
// vector.
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace qsim {

// ---------------------------------------------------------------- host: matrices
int gate_matrix(int kind, const double *p, const double *mat, double o[8])
{
    const double r2 = 0.70710678118654752440;
    const double th = p[0], ph = p[1], la = p[2];
    for (int k = 0; k < 8; ++k) o[k] = 0.0;
    switch (kind) {
    case SIM_GATE_U: for (int k = 0; k < 8; ++k) o[k] = mat[k]; return 0;
    case SIM_GATE_X: o[2] = 1; o[4] = 1; return 0;
    case SIM_GATE_Y: o[3] = -1; o[5] = 1; return 0;
    case SIM_GATE_Z: o[0] = 1; o[6] = -1; return 0;
    case SIM_GATE_H: o[0] = r2; o[2] = r2; o[4] = r2; o[6] = -r2; return 0;
    case SIM_GATE_S: o[0] = 1; o[7] = 1; return 0;
    case SIM_GATE_SDG: o[0] = 1; o[7] = -1; return 0;
    case SIM_GATE_T: o[0] = 1; o[6] = r2; o[7] = r2; return 0;
    case SIM_GATE_TDG: o[0] = 1; o[6] = r2; o[7] = -r2; return 0;
    case SIM_GATE_RX: {
        double c = std::cos(0.5 * th), s = std::sin(0.5 * th);
        o[0] = c; o[3] = -s; o[5] = -s; o[6] = c; return 0;
    }
    case SIM_GATE_RY: {
        double c = std::cos(0.5 * th), s = std::sin(0.5 * th);
        o[0] = c; o[2] = -s; o[4] = s; o[6] = c; return 0;
    }
    case SIM_GATE_RZ: {
        double c = std::cos(0.5 * th), s = std::sin(0.5 * th);
        o[0] = c; o[1] = -s; o[6] = c; o[7] = s; return 0;
    }
    case SIM_GATE_P: o[0] = 1; o[6] = std::cos(th); o[7] = std::sin(th); return 0;
    case SIM_GATE_U3: {
        double c = std::cos(0.5 * th), s = std::sin(0.5 * th);
        o[0] = c;
        o[2] = -std::cos(la) * s; o[3] = -std::sin(la) * s;
        o[4] = std::cos(ph) * s;  o[5] = std::sin(ph) * s;
        o[6] = std::cos(ph + la) * c; o[7] = std::sin(ph + la) * c;
        return 0;
    }
    default: return -1;
    }
}

int classify_matrix(const double m[8])
{
    const bool b0 = m[2] == 0 && m[3] == 0, c0 = m[4] == 0 && m[5] == 0;
    const bool a1 = m[0] == 1 && m[1] == 0, d1 = m[6] == 1 && m[7] == 0;
    const bool a0 = m[0] == 0 && m[1] == 0, d0 = m[6] == 0 && m[7] == 0;
    if (b0 && c0) {
        if (a1 && d1) return OP_IDENTITY;
        if (a1) return OP_DIAG_HI;
        return OP_DIAG;
    }
    if (a0 && d0) {
        const bool b1 = m[2] == 1 && m[3] == 0, c1 = m[4] == 1 && m[5] == 0;
        return (b1 && c1) ? OP_XPERM : OP_ANTIDIAG;
    }
    return OP_DENSE;
}

int validate_gate(int n, const sim_gate &g, std::string *why)
{
    auto bad = [&](const char *m) { if (why) *why = m; return -1; };
    if (g.kind >= SIM_GATE_CH_DEPOLARIZING && g.kind <= SIM_GATE_CH_PHASE_FLIP)
        return bad("noise channels apply to density-matrix handles only (sim_dm_apply_circuit)");
    if (g.kind < SIM_GATE_U || g.kind > SIM_GATE_SWAP) return bad("unknown gate kind");
    if (g.target < 0 || g.target >= n) return bad("target qubit out of range");
    if (g.n_controls < 0 || g.n_controls > 2) return bad("n_controls must be 0, 1 or 2");
    if (g.kind == SIM_GATE_SWAP) {
        if (g.target2 < 0 || g.target2 >= n) return bad("swap partner out of range");
        if (g.target2 == g.target) return bad("swap of a qubit with itself");
    }
    for (int c = 0; c < g.n_controls; ++c) {
        int q = g.controls[c];
        if (q < 0 || q >= n) return bad("control qubit out of range");
        if (q == g.target || (g.kind == SIM_GATE_SWAP && q == g.target2)) return bad("control equals a target");
        for (int d = 0; d < c; ++d)
            if (g.controls[d] == q) return bad("duplicate control qubit");
    }
    if (g.kind == SIM_GATE_U)
        for (int k = 0; k < 8; ++k)
            if (!std::isfinite(g.matrix[k])) return bad("non-finite matrix entry");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(g.params[k])) return bad("non-finite gate parameter");
    return 0;
}

PairGate make_pair_gate(const sim_gate &g)
{
    PairGate p{};
    p.target = g.target;
    p.target2 = g.target2;
    p.nctrl = g.n_controls;
    p.ctrl[0] = g.controls[0];
    p.ctrl[1] = g.controls[1];
    if (g.kind == SIM_GATE_SWAP) {
        p.op = OP_SWAP;
        return p;
    }
    gate_matrix(g.kind, g.params, g.matrix, p.m);
    p.op = classify_matrix(p.m);
    return p;
}

namespace {

struct PairArgs {
    uint64_t n_items;      // work items in the launch
    uint64_t set_mask;     // bits set on every base index (the controls)
    uint64_t lo_off;       // first amplitude = base | lo_off
    uint64_t hi_off;       // second amplitude = base | hi_off
    int npos;              // zero bits inserted at pos[0] < pos[1] < ...
    int pos[4];
};

template <typename R>
struct Coef { R ar, ai, br, bi, cr, ci, dr, di; };

__device__ __forceinline__ uint64_t insert_zeros(uint64_t w, const PairArgs &a)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k < a.npos) {
            const int p = a.pos[k];
            const uint64_t low = w & ((1ull << p) - 1ull);
            w = ((w >> p) << (p + 1)) | low;
        }
    }
    return w;
}

// the update of one amplitude pair (lo = v_a, hi = v_b)
template <int OP, typename R>
__device__ __forceinline__ void pair_update(R &lr, R &li, R &hr, R &hi, const Coef<R> &c)
{
    if (OP == OP_DENSE) {
        const R nlr = c.ar * lr - c.ai * li + (c.br * hr - c.bi * hi);
        const R nli = c.ar * li + c.ai * lr + (c.br * hi + c.bi * hr);
        const R nhr = c.cr * lr - c.ci * li + (c.dr * hr - c.di * hi);
        const R nhi = c.cr * li + c.ci * lr + (c.dr * hi + c.di * hr);
        lr = nlr; li = nli; hr = nhr; hi = nhi;
    } else if (OP == OP_DIAG) {
        const R nlr = c.ar * lr - c.ai * li, nli = c.ar * li + c.ai * lr;
        const R nhr = c.dr * hr - c.di * hi, nhi = c.dr * hi + c.di * hr;
        lr = nlr; li = nli; hr = nhr; hi = nhi;
    } else if (OP == OP_DIAG_HI) {
        const R nhr = c.dr * hr - c.di * hi, nhi = c.dr * hi + c.di * hr;
        hr = nhr; hi = nhi;
    } else if (OP == OP_ANTIDIAG) {
        const R nlr = c.br * hr - c.bi * hi, nli = c.br * hi + c.bi * hr;
        const R nhr = c.cr * lr - c.ci * li, nhi = c.cr * li + c.ci * lr;
        lr = nlr; li = nli; hr = nhr; hi = nhi;
    } else {  // OP_XPERM, OP_SWAP: pure exchange, bit-exact
        R t = lr; lr = hr; hr = t;
        t = li; li = hi; hi = t;
    }
}

template <typename R, int VEC> struct Vec;
template <> struct Vec<float, 1> { using T = float2; };
template <> struct Vec<float, 2> { using T = float4; };
template <> struct Vec<double, 1> { using T = double2; };

template <typename R, int VEC>
__device__ __forceinline__ typename Vec<R, VEC>::T ldv(const R *st, uint64_t amp)
{
    return *reinterpret_cast<const typename Vec<R, VEC>::T *>(st + 2 * amp);
}
template <typename R, int VEC>
__device__ __forceinline__ void stv(R *st, uint64_t amp, const typename Vec<R, VEC>::T &v)
{
    *reinterpret_cast<typename Vec<R, VEC>::T *>(st + 2 * amp) = v;
}

constexpr int kThreads = 256;

// Two separate vector accesses per item: the lo amplitudes at base | lo_off
// and the hi amplitudes at base | hi_off.  VEC neighbouring amplitudes per
// vector (all involved bits are >= log2(VEC)).
template <typename R, int VEC, int OP, int U>
__global__ void __launch_bounds__(kThreads) k_pair_split(R *__restrict__ st, PairArgs a, Coef<R> c)
{
    using V = typename Vec<R, VEC>::T;
    const uint64_t first = (uint64_t)blockIdx.x * (uint64_t)(kThreads * U) + threadIdx.x;
    V lo[U], hi[U];
    uint64_t base[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint64_t w = first + (uint64_t)u * kThreads;
        base[u] = ~0ull;
        if (w < a.n_items) {
            base[u] = insert_zeros(w * VEC, a) | a.set_mask;
            if (OP != OP_DIAG_HI) lo[u] = ldv<R, VEC>(st, base[u] | a.lo_off);
            hi[u] = ldv<R, VEC>(st, base[u] | a.hi_off);
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (base[u] == ~0ull) continue;
        if constexpr (VEC == 2) {
            float4 l = (OP != OP_DIAG_HI) ? lo[u] : make_float4(0, 0, 0, 0), h = hi[u];
            pair_update<OP, float>(l.x, l.y, h.x, h.y, c);
            pair_update<OP, float>(l.z, l.w, h.z, h.w, c);
            if (OP != OP_DIAG_HI) stv<R, VEC>(st, base[u] | a.lo_off, l);
            stv<R, VEC>(st, base[u] | a.hi_off, h);
        } else {
            V l = (OP != OP_DIAG_HI) ? lo[u] : V{}, h = hi[u];
            pair_update<OP, R>(l.x, l.y, h.x, h.y, c);
            if (OP != OP_DIAG_HI) stv<R, VEC>(st, base[u] | a.lo_off, l);
            stv<R, VEC>(st, base[u] | a.hi_off, h);
        }
    }
}

// complex64, target on bit 0: the pair (base, base + 1) is one 16-byte vector.
template <int OP, int U>
__global__ void __launch_bounds__(kThreads) k_pair_inner(float *__restrict__ st, PairArgs a, Coef<float> c)
{
    const uint64_t first = (uint64_t)blockIdx.x * (uint64_t)(kThreads * U) + threadIdx.x;
    float4 v[U];
    uint64_t base[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint64_t w = first + (uint64_t)u * kThreads;
        base[u] = ~0ull;
        if (w < a.n_items) {
            base[u] = insert_zeros(w, a) | a.set_mask;
            v[u] = ldv<float, 2>(st, base[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (base[u] == ~0ull) continue;
        float4 p = v[u];
        pair_update<OP, float>(p.x, p.y, p.z, p.w, c);
        stv<float, 2>(st, base[u], p);
    }
}

template <typename R>
Coef<R> make_coef(const double m[8])
{
    Coef<R> c;
    c.ar = (R)m[0]; c.ai = (R)m[1]; c.br = (R)m[2]; c.bi = (R)m[3];
    c.cr = (R)m[4]; c.ci = (R)m[5]; c.dr = (R)m[6]; c.di = (R)m[7];
    return c;
}

template <typename R, int VEC, int OP, int U>
cudaError_t go_split(qsim_state *s, const PairArgs &a, const Coef<R> &c)
{
    const uint64_t per = (uint64_t)kThreads * U;
    const uint64_t blocks = (a.n_items + per - 1) / per;
    k_pair_split<R, VEC, OP, U><<<(unsigned)blocks, kThreads, 0, s->stream>>>((R *)s->amps, a, c);
    return cudaSuccess;
}

template <int OP>
cudaError_t go_inner(qsim_state *s, const PairArgs &a, const Coef<float> &c)
{
    constexpr int U = 4;
    const uint64_t per = (uint64_t)kThreads * U;
    const uint64_t blocks = (a.n_items + per - 1) / per;
    k_pair_inner<OP, U><<<(unsigned)blocks, kThreads, 0, s->stream>>>((float *)s->amps, a, c);
    return cudaSuccess;
}

template <typename R, int VEC, int U>
void dispatch_split(qsim_state *s, int op, const PairArgs &a, const Coef<R> &c)
{
    switch (op) {
    case OP_DENSE: go_split<R, VEC, OP_DENSE, U>(s, a, c); break;
    case OP_DIAG: go_split<R, VEC, OP_DIAG, U>(s, a, c); break;
    case OP_DIAG_HI: go_split<R, VEC, OP_DIAG_HI, U>(s, a, c); break;
    case OP_ANTIDIAG: go_split<R, VEC, OP_ANTIDIAG, U>(s, a, c); break;
    default: go_split<R, VEC, OP_XPERM, U>(s, a, c); break;   // XPERM and SWAP
    }
}

void dispatch_inner(qsim_state *s, int op, const PairArgs &a, const Coef<float> &c)
{
    switch (op) {
    case OP_DENSE: go_inner<OP_DENSE>(s, a, c); break;
    case OP_DIAG: go_inner<OP_DIAG>(s, a, c); break;
    case OP_DIAG_HI: go_inner<OP_DIAG_HI>(s, a, c); break;
    case OP_ANTIDIAG: go_inner<OP_ANTIDIAG>(s, a, c); break;
    default: go_inner<OP_XPERM>(s, a, c); break;
    }
}

int op_class(int op)
{
    switch (op) {
    case OP_DENSE: return KC_DENSE;
    case OP_DIAG: case OP_DIAG_HI: return KC_DIAG;
    case OP_SWAP: return KC_SWAP;
    default: return KC_PERM;
    }
}

}  // namespace

static int launch_pair_impl(qsim_state *s, const PairGate &g, uint64_t cm);

int launch_pair_gate(qsim_state *s, const PairGate &g)
{
    uint64_t cm = 0;
    for (int k = 0; k < g.nctrl; ++k) cm |= 1ull << g.ctrl[k];
    return launch_pair_impl(s, g, cm);
}

int launch_sgate(qsim_state *s, const SGate &sg)
{
    PairGate g{};
    g.op = sg.op;
    g.target = sg.target;
    g.target2 = -1;
    g.nctrl = 0;
    memcpy(g.m, sg.m, sizeof g.m);
    return launch_pair_impl(s, g, sg.ctrl);
}

static int launch_pair_impl(qsim_state *s, const PairGate &g, uint64_t cm)
{
    if (g.op == OP_IDENTITY) return SIM_OK;
    if (__builtin_popcountll(cm) > 3) return fail(SIM_EUNSUPPORTED, "per-gate launch: at most 3 controls");
    PairArgs a{};
    int pos[4], np = 0;
    pos[np++] = g.target;
    if (g.op == OP_SWAP) pos[np++] = g.target2;
    for (int q = 0; q < 64 && np < 4; ++q)
        if ((cm >> q) & 1) pos[np++] = q;
    for (int i = 1; i < np; ++i)            // insertion sort, ascending
        for (int j = i; j > 0 && pos[j - 1] > pos[j]; --j) {
            int t = pos[j]; pos[j] = pos[j - 1]; pos[j - 1] = t;
        }
    a.npos = np;
    for (int k = 0; k < np; ++k) a.pos[k] = pos[k];
    a.set_mask = cm;
    if (g.op == OP_SWAP) {
        a.lo_off = 1ull << g.target;     // bit target = 1, bit target2 = 0
        a.hi_off = 1ull << g.target2;    // bit target = 0, bit target2 = 1
    } else {
        a.lo_off = 0;
        a.hi_off = 1ull << g.target;
    }
    const uint64_t bases = 1ull << (s->n - np);
    // amplitudes the gate must change: 2 per base (1 for a phase on |1>), read + written
    const double amp = (s->dtype == SIM_C128) ? 16.0 : 8.0;
    const double touched = (double)bases * ((g.op == OP_DIAG_HI) ? 1.0 : 2.0);
    double flops = 0.0;
    if (g.op == OP_DENSE) flops = 16.0 * touched;
    else if (g.op == OP_DIAG || g.op == OP_ANTIDIAG) flops = 6.0 * touched;
    else if (g.op == OP_DIAG_HI) flops = (g.m[6] == -1.0 && g.m[7] == 0.0) ? 0.0 : 6.0 * touched;
    launch_begin(s, op_class(g.op), 2.0 * touched * amp, flops);
    if (s->dtype == SIM_C128) {
        a.n_items = bases;
        dispatch_split<double, 1, 2>(s, g.op, a, make_coef<double>(g.m));
    } else {
        Coef<float> c = make_coef<float>(g.m);
        if (pos[0] >= 1) {
            a.n_items = bases / 2;
            dispatch_split<float, 2, 4>(s, g.op, a, c);
        } else if (g.op != OP_SWAP && g.target == 0) {
            a.n_items = bases;
            dispatch_inner(s, g.op, a, c);
        } else {
            a.n_items = bases;
            dispatch_split<float, 1, 4>(s, g.op, a, c);
        }
    }
    return launch_end(s, "pair gate");
}

}  // namespace qsim
