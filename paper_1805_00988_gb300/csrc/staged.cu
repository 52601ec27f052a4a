// staged.cu -- multi-gate tile passes: one HBM read + write of the state
// applies a whole run of gates.
//
// Algorithm 1 (§2.3) touches the full state once per gate.  Consecutive gates
// whose non-diagonal qubits all lie in one qubit set Q can instead be applied
// tile by tile: a tile is the 2^M amplitudes that share the bits of every
// qubit outside Q, so a gate on a qubit of Q only pairs amplitudes inside one
// tile.  Q always holds the low qubits 0..4 (so a tile is made of contiguous
// 32-amplitude chunks) plus M - 5 further qubits chosen per pass.  Diagonal
// gates (Z, S, T, P, RZ, CZ, CP, ...) and controls never need their qubit in
// Q: outside Q the bit is constant over the tile.
//
// Inside a CTA the tile lives in registers: with 256 threads each thread holds
// 2^(M-8) amplitudes.  A register layout assigns the tile's local bits to
// register bits and thread bits; a gate whose target is a register bit is
// applied by each thread alone.  Layouts change through shared memory (one
// store + one load of the tile, XOR-swizzled so every layout is free of bank
// conflicts).  The host planner (below) forms the passes, orders the gates of
// a pass to need few layout changes, and encodes each gate as register /
// thread / tile masks for the layout current at that point.
#include <algorithm>
#include <cstring>
#include <vector>

#include "tile.cuh"

namespace qsim {

namespace {

// complex64 tiles of up to 12 qubits hold 16 amplitudes a thread and fit 80
// registers: three CTAs per SM; 13-qubit and complex128 tiles two.  kRamp:
// the variant that also runs SK_RAMP ops, launched for the passes that have
// them.
template <typename R, int M, bool kRamp>
__global__ void __launch_bounds__(kThr, (sizeof(R) == 4 && M <= 12 ? 3 : 2))
k_staged(R *__restrict__ st, const StOp<R> *__restrict__ ops, int nops,
                                                   TileGeom geo)
{
    constexpr int VEC = (sizeof(R) == 4) ? 2 : 1;
    constexpr int RB = M - kThrBits;
    constexpr int RA = 1 << RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sm = reinterpret_cast<R *>(smem_raw);
    const int tid = threadIdx.x;

    const uint64_t tile = (uint64_t)blockIdx.x;
    uint64_t base = 0;
    for (int i = 0; i < geo.n_outer; ++i) base |= ((tile >> i) & 1ull) << geo.outer_pos[i];

    // global offsets in the I/O layout: the thread's offset and one per
    // register bit.  They are formed again for the store (from inputs the
    // compiler cannot prove equal) instead of being held live across the
    // gate sequence, which would spill at two CTAs per SM.
    uint64_t toff, roff[RB];
    auto io_offsets = [&](int t, uint64_t b0) {
        toff = b0;
#pragma unroll
        for (int i = 0; i < kThrBits; ++i) {
            const int b = thr_local(M, RB, VEC, 0, i);
            const uint64_t g = (b < kLow) ? (1ull << b) : (1ull << geo.hpos[b - kLow]);
            if ((t >> i) & 1) toff |= g;
        }
#pragma unroll
        for (int j = 0; j < RB; ++j) {
            const int b = reg_local(M, RB, VEC, 0, j);
            roff[j] = (b < kLow) ? (1ull << b) : (1ull << geo.hpos[b - kLow]);
        }
    };
    io_offsets(tid, base);

    Regs<R, RA> v;
    if constexpr (VEC == 2) {
#pragma unroll
        for (int k = 0; k < RA; k += 2) {
            uint64_t g = toff;
#pragma unroll
            for (int j = 1; j < RB; ++j)
                if ((k >> j) & 1) g |= roff[j];
            const float4 t = *reinterpret_cast<const float4 *>(st + 2 * g);
            v.set2(k >> 1, t.x, t.y, t.z, t.w);
        }
    } else {
#pragma unroll
        for (int k = 0; k < RA; ++k) {
            uint64_t g = toff;
#pragma unroll
            for (int j = 0; j < RB; ++j)
                if ((k >> j) & 1) g |= roff[j];
            const double2 t = *reinterpret_cast<const double2 *>(st + 2 * g);
            v.setr(k, (R)t.x);
            v.seti(k, (R)t.y);
        }
    }

    apply_ops<R, M, kRamp>(v, ops, nops, base, tid, sm,
                    reinterpret_cast<StOp<R> *>(smem_raw + ((size_t)1 << M) * 2 * sizeof(R)));
    {
        int t2 = tid;
        uint64_t b2 = base;
        asm volatile("" : "+r"(t2), "+l"(b2));
        io_offsets(t2, b2);
    }
    // the planner always ends a pass in layout 0
    if constexpr (VEC == 2) {
#pragma unroll
        for (int k = 0; k < RA; k += 2) {
            uint64_t g = toff;
#pragma unroll
            for (int j = 1; j < RB; ++j)
                if ((k >> j) & 1) g |= roff[j];
            *reinterpret_cast<float4 *>(st + 2 * g) = make_float4(v.getr(k), v.geti(k), v.getr(k + 1), v.geti(k + 1));
        }
    } else {
#pragma unroll
        for (int k = 0; k < RA; ++k) {
            uint64_t g = toff;
#pragma unroll
            for (int j = 0; j < RB; ++j)
                if ((k >> j) & 1) g |= roff[j];
            *reinterpret_cast<double2 *>(st + 2 * g) = make_double2((double)v.getr(k), (double)v.geti(k));
        }
    }
}

template <typename R, int M, bool kRamp>
int launch_staged_v(qsim_state *s, const StOp<R> *dops, int nops, const TileGeom &geo, double flops)
{
    const size_t smem = ((size_t)1 << M) * 2 * sizeof(R) + op_stage_bytes<R>();
    // set on every launch: the attribute belongs to the current device's
    // context, and the call costs a microsecond against a multi-ms pass
    QSIM_CUDA(cudaFuncSetAttribute(k_staged<R, M, kRamp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const uint64_t tiles = 1ull << (s->n - M);
    launch_begin(s, KC_STAGED, 2.0 * (double)s->bytes, flops);
    k_staged<R, M, kRamp><<<(unsigned)tiles, kThr, smem, s->stream>>>((R *)s->amps, dops, nops, geo);
    return launch_end(s, "staged pass");
}

template <typename R, int M>
int launch_staged(qsim_state *s, const StOp<R> *dops, int nops, const TileGeom &geo, double flops, bool ramp)
{
    return ramp ? launch_staged_v<R, M, true>(s, dops, nops, geo, flops)
                : launch_staged_v<R, M, false>(s, dops, nops, geo, flops);
}

template <typename R>
int run_staged(qsim_state *s, const std::vector<SGate> &g, int M)
{
    const int VEC = sizeof(R) == 4 ? 2 : 1;
    std::vector<Pass> passes = form_passes(g, s->n, M);
    PlanBuilder<R> pb{s->n, M, M - kThrBits, VEC, {}, {}, 0};
    std::vector<int> counts;
    std::vector<double> pflops;
    std::vector<char> ramp;
    for (const Pass &ps : passes) {
        const size_t first = pb.ops.size();
        counts.push_back(pb.schedule(ps, g));
        bool r = false;
        for (size_t k = first; k < pb.ops.size() && !r; ++k) r = pb.ops[k].kind == SK_RAMP;
        ramp.push_back(r);
        double f = 0.0;
        for (int m : ps.members) f += sgate_flops(g[m], s->n);
        pflops.push_back(f);
    }
    const size_t bytes = pb.ops.size() * sizeof(StOp<R>);
    if (int rc = ensure_host_pinned(&s->host_ops, &s->host_ops_bytes, bytes)) return rc;
    if (int rc = ensure_device(s, &s->dev_ops, &s->dev_ops_bytes, bytes)) return rc;
    memcpy(s->host_ops, pb.ops.data(), bytes);
    QSIM_CUDA(cudaMemcpyAsync(s->dev_ops, s->host_ops, bytes, cudaMemcpyHostToDevice, s->stream));
    const StOp<R> *dops = (const StOp<R> *)s->dev_ops;
    size_t off = 0;
    for (size_t p = 0; p < passes.size(); ++p) {
        TileGeom geo;
        memset(&geo, 0, sizeof geo);
        uint64_t q = (1ull << kLow) - 1ull;
        for (size_t i = 0; i < passes[p].high.size(); ++i) {
            geo.hpos[i] = passes[p].high[i];
            q |= 1ull << passes[p].high[i];
        }
        for (int b = 0; b < s->n; ++b)
            if (!((q >> b) & 1)) geo.outer_pos[geo.n_outer++] = b;
        int rc;
        switch (M) {
        case 11: rc = launch_staged<R, 11>(s, dops + off, counts[p], geo, pflops[p], ramp[p]); break;
        case 12: rc = launch_staged<R, 12>(s, dops + off, counts[p], geo, pflops[p], ramp[p]); break;
        case 13:
            if constexpr (sizeof(R) == 4) rc = launch_staged<R, 13>(s, dops + off, counts[p], geo, pflops[p], ramp[p]);
            else rc = fail(SIM_EINVAL, "staged: complex128 tiles are at most 12 qubits");
            break;
        default: rc = fail(SIM_EINVAL, "staged: unsupported tile size");
        }
        if (rc) return rc;
        off += counts[p];
    }
    // the pinned staging buffer is reused by the next call: wait for the copy
    QSIM_CUDA(cudaStreamSynchronize(s->stream));
    return SIM_OK;
}

}  // namespace

int describe_staged(int n, int dtype, const sim_gate *gates, size_t n_gates, int tile_qubits, int64_t *passes,
                    int64_t *ops, int64_t *layout_changes, int32_t *order, size_t order_cap, size_t *order_len)
{
    const bool c128 = dtype == SIM_C128;
    int M = tile_qubits ? tile_qubits : (c128 ? 11 : 13);
    if (M > n || M < 11 || M > (c128 ? 12 : 13)) return fail(SIM_EINVAL, "describe: no staged tile fits");
    std::vector<SGate> g;
    lower_gates(gates, n_gates, &g);
    std::vector<Pass> ps = form_passes(g, n, M);
    PlanBuilder<double> pb{n, M, M - kThrBits, c128 ? 1 : 2, {}, {}, 0};
    for (const Pass &p : ps) pb.schedule(p, g);
    if (passes) *passes = (int64_t)ps.size();
    if (ops) *ops = (int64_t)(pb.ops.size() - pb.filler);   // a phase ramp counts once
    if (layout_changes) *layout_changes = pb.layout_changes;
    if (order_len) *order_len = pb.order.size();
    if (order)
        for (size_t i = 0; i < pb.order.size() && i < order_cap; ++i) order[i] = pb.order[i];
    return SIM_OK;
}

int encode_staged(int n, int dtype, const sim_gate *gates, size_t n_gates, int tile_qubits, sim_tile_op *ops,
                  size_t ops_cap, int32_t *info, size_t info_cap, size_t *n_ops, size_t *n_passes)
{
    const bool c128 = dtype == SIM_C128;
    int M = tile_qubits ? tile_qubits : (c128 ? 11 : 13);
    if (M > n || M < 11 || M > (c128 ? 12 : 13)) return fail(SIM_EINVAL, "encode: no staged tile fits");
    std::vector<SGate> g;
    lower_gates(gates, n_gates, &g);
    std::vector<Pass> ps = form_passes(g, n, M);
    PlanBuilder<double> pb{n, M, M - kThrBits, c128 ? 1 : 2, {}, {}, 0};
    std::vector<size_t> first;
    for (const Pass &p : ps) {
        first.push_back(pb.ops.size());
        pb.schedule(p, g);
    }
    if (n_ops) *n_ops = pb.ops.size();
    if (n_passes) *n_passes = ps.size();
    for (size_t k = 0; k < pb.ops.size() && k < ops_cap && ops; ++k) {
        const StOp<double> &o = pb.ops[k];
        sim_tile_op &t = ops[k];
        t.kind = o.kind;
        t.arg = o.arg;
        t.thr_c = o.thr_c;
        t.plain = o.plain;
        t.out_c = o.out_c;
        t.km_c = o.km_c;
        t.km_t = o.km_t;
        t.thr_t = o.thr_t;
        t.pad = 0;
        t.out_t = o.out_t;
        for (int j = 0; j < 8; ++j) t.m[j] = o.m[j];
    }
    for (size_t p = 0; p < ps.size() && info && (p + 1) * SIM_TILE_PASS_INFO <= info_cap; ++p) {
        int32_t *r = info + p * SIM_TILE_PASS_INFO;
        for (int j = 0; j < SIM_TILE_PASS_INFO; ++j) r[j] = 0;
        r[0] = (int32_t)first[p];
        r[1] = (int32_t)((p + 1 < ps.size() ? first[p + 1] : pb.ops.size()) - first[p]);
        r[2] = M;
        r[3] = M - kThrBits;
        r[4] = c128 ? 1 : 2;
        r[5] = (int32_t)ps[p].high.size();
        for (size_t i = 0; i < ps[p].high.size() && i < 16; ++i) r[6 + i] = ps[p].high[i];
    }
    return SIM_OK;
}

int apply_circuit_staged(qsim_state *s, const sim_gate *gates, size_t n_gates, const sim_plan_opts &o)
{
    const bool c128 = s->dtype == SIM_C128;
    int M = o.tile_qubits ? o.tile_qubits : (c128 ? 11 : 13);
    if (M > s->n) M = (s->n >= 11) ? 11 : 0;
    if (c128 && M > 12) M = 12;
    if (M != 0 && (M < 11 || M > 13)) return fail(SIM_EINVAL, "staged: tile_qubits must be 11, 12 or 13");
    if (M == 0) {
        // the state is smaller than a tile: one launch per gate
        for (size_t k = 0; k < n_gates; ++k)
            if (int rc = launch_pair_gate(s, make_pair_gate(gates[k]))) return rc;
        return SIM_OK;
    }
    std::vector<SGate> g;
    lower_gates(gates, n_gates, &g);
    if (g.empty()) return SIM_OK;
    return c128 ? run_staged<double>(s, g, M) : run_staged<float>(s, g, M);
}

}  // namespace qsim
