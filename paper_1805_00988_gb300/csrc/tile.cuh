// tile.cuh -- the register-resident tile machinery shared by the staged
// pass kernel and the batched persistent kernel: register layouts, the
// encoded gate ops, their application to a tile, and the host pass planner.
// See staged.cu for the design.
#pragma once

#include <complex>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace qsim {
namespace {


constexpr int kLow = 5;          // qubits 0..4 are local bits 0..4 of every tile
constexpr int kThr = 256;        // threads per CTA
constexpr int kThrBits = 8;

enum StKind { SK_LAYOUT = 0, SK_DENSE, SK_ANTI, SK_XPERM, SK_DIAG, SK_PHASE, SK_NEG, SK_RAMP, SK_NOP };

// SK_RAMP: a run of controlled phases that share one qubit q, each pairing q
// with a tile-local qubit m (phase f_m when both bits are 1), applied at
// once: amplitudes whose q bit is 1 are multiplied by the product of f_m over
// the local bits m that are 1 -- the product over the thread's thread bits
// times the product over the register's register bits.  The host tabulates
// both: entry k < RA is register k's product, entries RA + x and RA + 16 + y
// the products over thread bits 0..3 set in x and 4..7 set in y, so a thread
// forms its factor from two entries and each register needs one more.  Entry
// e sits in record e / 4 of the op, coefficient slots 2 (e % 4) and
// 2 (e % 4) + 1; the first record also carries q as a diagonal op's target
// (km_t / thr_t / out_t).  The other records, and the padding that keeps a
// ramp inside one staged chunk of kOpChunk ops, are SK_NOP records.
__host__ __device__ constexpr int ramp_records(int RA) { return (RA + 32 + 3) / 4; }
static_assert(kThrBits == 8, "ramp tables cover thread bits as two groups of four");

template <typename R>
struct __align__(16) StOp {
    int32_t kind;      // StKind
    int32_t arg;       // exchange ops: register bit of the target; SK_LAYOUT: new layout
    uint32_t thr_c;    // thread bits that must be 1
    int32_t plain;     // exchange ops: no condition of any kind
    uint64_t out_c;    // global bits (outside the tile) that must be 1
    uint64_t km_c;     // bit k: register k satisfies the register-bit conditions
    uint64_t km_t;     // diagonal ops, bit k: the target bit of register k is 1
    uint32_t thr_t;    // diagonal ops: thread bit of the target (0 if not a thread bit)
    uint32_t pad;
    uint64_t out_t;    // diagonal ops: global bit of the target (0 if inside the tile)
    R m[8];            // A, B, C, D
};

// ---------------------------------------------------------------- layouts
// VEC = 2 for complex64 (the I/O layout keeps local bit 0 in registers so a
// thread loads two neighbouring amplitudes as one 16-byte vector), 1 for
// complex128.  Layout 0 is the I/O layout; layouts 1.. put windows of RB
// consecutive local bits into registers.
__host__ __device__ constexpr int n_layouts(int M, int RB) { return 1 + (M - RB + RB - 1) / RB; }

__host__ __device__ constexpr int reg_local(int M, int RB, int VEC, int l, int j)
{
    if (l == 0) return (VEC == 2) ? (j == 0 ? 0 : M - RB + j) : (M - RB + j);
    int s = (VEC == 2 ? 1 : 0) + RB * (l - 1);
    if (s > M - RB) s = M - RB;
    return s + j;
}

__host__ __device__ constexpr bool is_reg(int M, int RB, int VEC, int l, int b)
{
    for (int j = 0; j < RB; ++j)
        if (reg_local(M, RB, VEC, l, j) == b) return true;
    return false;
}

__host__ __device__ constexpr int thr_local(int M, int RB, int VEC, int l, int i)
{
    int c = 0;
    for (int b = 0; b < M; ++b)
        if (!is_reg(M, RB, VEC, l, b)) {
            if (c == i) return b;
            ++c;
        }
    return -1;
}

__host__ __device__ constexpr int reg_part(int M, int RB, int VEC, int l, int k)
{
    int x = 0;
    for (int j = 0; j < RB; ++j)
        if ((k >> j) & 1) x |= 1 << reg_local(M, RB, VEC, l, j);
    return x;
}

// shared-memory slot of local index x (bank-conflict-free for every layout)
template <int RB, int VEC>
__host__ __device__ constexpr int swz(int x)
{
    return (VEC == 2) ? (x ^ (((x >> (RB + 1)) & 7) << 1)) : (x ^ ((x >> RB) & 7));
}

struct TileGeom {
    int n_outer;
    int outer_pos[40];   // global qubit of outer bit i (ascending)
    int hpos[16];        // global qubit of local bit kLow + i
};

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

// ---------------------------------------------------------------- registers
// Amplitudes of a thread.  complex64 keeps them as float2 packs along
// register bit 0 so that two amplitude pairs go through one packed FP32x2
// instruction (fma.rn.f32x2); complex128 keeps plain doubles.
template <typename R, int RA> struct Regs;
template <int RA> struct Regs<float, RA> {
    // pack p = (amplitude 2p, amplitude 2p + 1) in one float2 register pair
    float2 r[RA / 2], i[RA / 2];
    __device__ __forceinline__ float getr(int k) const { return (k & 1) ? r[k >> 1].y : r[k >> 1].x; }
    __device__ __forceinline__ float geti(int k) const { return (k & 1) ? i[k >> 1].y : i[k >> 1].x; }
    __device__ __forceinline__ void setr(int k, float v)
    {
        if (k & 1) r[k >> 1].y = v; else r[k >> 1].x = v;
    }
    __device__ __forceinline__ void seti(int k, float v)
    {
        if (k & 1) i[k >> 1].y = v; else i[k >> 1].x = v;
    }
    __device__ __forceinline__ void set2(int p, float r0, float i0, float r1, float i1)
    {
        r[p] = make_float2(r0, r1);
        i[p] = make_float2(i0, i1);
    }
};
template <int RA> struct Regs<double, RA> {
    double r[RA], i[RA];
    __device__ __forceinline__ double getr(int k) const { return r[k]; }
    __device__ __forceinline__ double geti(int k) const { return i[k]; }
    __device__ __forceinline__ void setr(int k, double v) { r[k] = v; }
    __device__ __forceinline__ void seti(int k, double v) { i[k] = v; }
};

template <typename R>
struct CoefS { R ar, ai, br, bi, cr, ci, dr, di; };

// packed FP32x2 arithmetic (sm_100+ builtins on float2 register pairs)
struct PCoef { float2 ar, ai, nai, br, bi, nbi, cr, ci, nci, dr, di, ndi; };

__device__ __forceinline__ PCoef make_pcoef(const CoefS<float> &c)
{
    PCoef p;
    p.ar = make_float2(c.ar, c.ar); p.ai = make_float2(c.ai, c.ai); p.nai = make_float2(-c.ai, -c.ai);
    p.br = make_float2(c.br, c.br); p.bi = make_float2(c.bi, c.bi); p.nbi = make_float2(-c.bi, -c.bi);
    p.cr = make_float2(c.cr, c.cr); p.ci = make_float2(c.ci, c.ci); p.nci = make_float2(-c.ci, -c.ci);
    p.dr = make_float2(c.dr, c.dr); p.di = make_float2(c.di, c.di); p.ndi = make_float2(-c.di, -c.di);
    return p;
}

// two amplitude pairs at once: lanes x / y are independent pairs
template <int KIND>
__device__ __forceinline__ void pupd(float2 &lr, float2 &li, float2 &hr, float2 &hi, const PCoef &c)
{
    if (KIND == SK_DENSE) {
        const float2 nlr = __ffma2_rn(c.ar, lr, __ffma2_rn(c.nai, li, __ffma2_rn(c.br, hr, __fmul2_rn(c.nbi, hi))));
        const float2 nli = __ffma2_rn(c.ar, li, __ffma2_rn(c.ai, lr, __ffma2_rn(c.br, hi, __fmul2_rn(c.bi, hr))));
        const float2 nhr = __ffma2_rn(c.cr, lr, __ffma2_rn(c.nci, li, __ffma2_rn(c.dr, hr, __fmul2_rn(c.ndi, hi))));
        const float2 nhi = __ffma2_rn(c.cr, li, __ffma2_rn(c.ci, lr, __ffma2_rn(c.dr, hi, __fmul2_rn(c.di, hr))));
        lr = nlr; li = nli; hr = nhr; hi = nhi;
    } else if (KIND == SK_ANTI) {
        const float2 nlr = __ffma2_rn(c.br, hr, __fmul2_rn(c.nbi, hi));
        const float2 nli = __ffma2_rn(c.br, hi, __fmul2_rn(c.bi, hr));
        const float2 nhr = __ffma2_rn(c.cr, lr, __fmul2_rn(c.nci, li));
        const float2 nhi = __ffma2_rn(c.cr, li, __fmul2_rn(c.ci, lr));
        lr = nlr; li = nli; hr = nhr; hi = nhi;
    } else {
        float2 t = lr; lr = hr; hr = t;
        t = li; li = hi; hi = t;
    }
}

template <int KIND, typename R>
__device__ __forceinline__ void xupd(R &lr, R &li, R &hr, R &hi, const CoefS<R> &c)
{
    if (KIND == SK_DENSE) {
        const R nlr = c.ar * lr - c.ai * li + (c.br * hr - c.bi * hi);
        const R nli = c.ar * li + c.ai * lr + (c.br * hi + c.bi * hr);
        const R nhr = c.cr * lr - c.ci * li + (c.dr * hr - c.di * hi);
        const R nhi = c.cr * li + c.ci * lr + (c.dr * hi + c.di * hr);
        lr = nlr; li = nli; hr = nhr; hi = nhi;
    } else if (KIND == SK_ANTI) {
        const R nlr = c.br * hr - c.bi * hi, nli = c.br * hi + c.bi * hr;
        const R nhr = c.cr * lr - c.ci * li, nhi = c.cr * li + c.ci * lr;
        lr = nlr; li = nli; hr = nhr; hi = nhi;
    } else {  // SK_XPERM: exact exchange
        R t = lr; lr = hr; hr = t;
        t = li; li = hi; hi = t;
    }
}

// Exchange op on register bit J.  PLAIN: no condition at all.  Otherwise the
// amplitude pair (k, k | 2^J) is updated when bit k of `act` is set.
template <int J, int KIND, bool PLAIN, typename R, int RA>
__device__ __forceinline__ void xop(Regs<R, RA> &v, uint64_t act, const CoefS<R> &c)
{
    constexpr int RB = __builtin_ctz(RA);
    if constexpr (J < RB) {
        if constexpr (sizeof(R) == 4 && J >= 1) {
            // packed: packs p and p | 2^(J-1) hold pairs (2p, 2p + 2^J) and (2p + 1, 2p + 1 + 2^J)
            const PCoef pc = make_pcoef(c);
#pragma unroll
            for (int p = 0; p < RA / 2; ++p) {
                if (p & (1 << (J - 1))) continue;
                const int q = p | (1 << (J - 1));
                if (PLAIN) {
                    pupd<KIND>(v.r[p], v.i[p], v.r[q], v.i[q], pc);
                } else {
                    const bool a0 = (act >> (2 * p)) & 1, a1 = (act >> (2 * p + 1)) & 1;
                    if (a0 && a1) {
                        pupd<KIND>(v.r[p], v.i[p], v.r[q], v.i[q], pc);
                    } else if (a0 || a1) {
                        const int k = 2 * p + (a0 ? 0 : 1), k1 = 2 * q + (a0 ? 0 : 1);
                        R lr = v.getr(k), li = v.geti(k), hr = v.getr(k1), hi = v.geti(k1);
                        xupd<KIND, R>(lr, li, hr, hi, c);
                        v.setr(k, lr); v.seti(k, li); v.setr(k1, hr); v.seti(k1, hi);
                    }
                }
            }
        } else if constexpr (sizeof(R) == 4 && J == 0) {
            // packed, the pair inside one pack: pack p = (amplitude 2p, 2p + 1)
            const float2 q1 = make_float2(c.ar, c.dr), q2 = make_float2(c.br, c.cr);
            const float2 q3 = make_float2(-c.ai, -c.di), q4 = make_float2(-c.bi, -c.ci);
            const float2 q5 = make_float2(c.ai, c.di), q6 = make_float2(c.bi, c.ci);
#pragma unroll
            for (int p = 0; p < RA / 2; ++p) {
                if (!PLAIN && !((act >> (2 * p)) & 1)) continue;
                const float2 R0 = v.r[p], I0 = v.i[p];
                const float2 Rs = make_float2(R0.y, R0.x), Is = make_float2(I0.y, I0.x);
                if (KIND == SK_DENSE) {
                    v.r[p] = __ffma2_rn(q1, R0, __ffma2_rn(q2, Rs, __ffma2_rn(q3, I0, __fmul2_rn(q4, Is))));
                    v.i[p] = __ffma2_rn(q1, I0, __ffma2_rn(q2, Is, __ffma2_rn(q5, R0, __fmul2_rn(q6, Rs))));
                } else if (KIND == SK_ANTI) {
                    v.r[p] = __ffma2_rn(q2, Rs, __fmul2_rn(q4, Is));
                    v.i[p] = __ffma2_rn(q2, Is, __fmul2_rn(q6, Rs));
                } else {
                    v.r[p] = Rs;
                    v.i[p] = Is;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < RA; ++k) {
                if (k & (1 << J)) continue;
                const int k1 = k | (1 << J);
                if (PLAIN || ((act >> k) & 1)) {
                    R lr = v.getr(k), li = v.geti(k), hr = v.getr(k1), hi = v.geti(k1);
                    xupd<KIND, R>(lr, li, hr, hi, c);
                    v.setr(k, lr); v.seti(k, li); v.setr(k1, hr); v.seti(k1, hi);
                }
            }
        }
    }
}

template <int KIND, bool PLAIN, typename R, int RA>
__device__ __forceinline__ void xdispatch(int j, Regs<R, RA> &v, uint64_t act, const CoefS<R> &c)
{
    switch (j) {
    case 0: xop<0, KIND, PLAIN>(v, act, c); break;
    case 1: xop<1, KIND, PLAIN>(v, act, c); break;
    case 2: xop<2, KIND, PLAIN>(v, act, c); break;
    case 3: xop<3, KIND, PLAIN>(v, act, c); break;
    case 4: xop<4, KIND, PLAIN>(v, act, c); break;
    case 5: xop<5, KIND, PLAIN>(v, act, c); break;
    default: break;
    }
}

template <int M, int RB, int VEC, int L, typename R, int RA>
__device__ __forceinline__ void store_layout(Regs<R, RA> &v, R *sm, int tid)
{
    if constexpr (L < n_layouts(M, RB)) {
        int tp = 0;
#pragma unroll
        for (int i = 0; i < kThrBits; ++i) tp |= ((tid >> i) & 1) << thr_local(M, RB, VEC, L, i);
        const int tps = swz<RB, VEC>(tp);   // swz is linear over XOR: swz(tp ^ r) = swz(tp) ^ swz(r)
        if constexpr (VEC == 2 && L == 0) {
#pragma unroll
            for (int k = 0; k < RA; k += 2) {
                const int p = tps ^ swz<RB, VEC>(reg_part(M, RB, VEC, L, k));
                *reinterpret_cast<float4 *>(sm + 2 * p) = make_float4(v.getr(k), v.geti(k), v.getr(k + 1), v.geti(k + 1));
            }
        } else {
#pragma unroll
            for (int k = 0; k < RA; ++k) {
                const int p = tps ^ swz<RB, VEC>(reg_part(M, RB, VEC, L, k));
                typename V2<R>::T t;
                t.x = v.getr(k);
                t.y = v.geti(k);
                *reinterpret_cast<typename V2<R>::T *>(sm + 2 * p) = t;
            }
        }
    }
}

template <int M, int RB, int VEC, int L, typename R, int RA>
__device__ __forceinline__ void load_layout(Regs<R, RA> &v, const R *sm, int tid)
{
    if constexpr (L < n_layouts(M, RB)) {
        int tp = 0;
#pragma unroll
        for (int i = 0; i < kThrBits; ++i) tp |= ((tid >> i) & 1) << thr_local(M, RB, VEC, L, i);
        const int tps = swz<RB, VEC>(tp);   // swz is linear over XOR: swz(tp ^ r) = swz(tp) ^ swz(r)
        if constexpr (VEC == 2 && L == 0) {
#pragma unroll
            for (int k = 0; k < RA; k += 2) {
                const int p = tps ^ swz<RB, VEC>(reg_part(M, RB, VEC, L, k));
                const float4 t = *reinterpret_cast<const float4 *>(sm + 2 * p);
                v.set2(k >> 1, t.x, t.y, t.z, t.w);
            }
        } else {
#pragma unroll
            for (int k = 0; k < RA; ++k) {
                const int p = tps ^ swz<RB, VEC>(reg_part(M, RB, VEC, L, k));
                const typename V2<R>::T t = *reinterpret_cast<const typename V2<R>::T *>(sm + 2 * p);
                v.setr(k, t.x);
                v.seti(k, t.y);
            }
        }
    }
}

// Sign flips (CZ, Z, CCZ) commute with every diagonal op, so they are
// collected in a per-thread mask (bit k: negate register k) and applied only
// before the next op that mixes registers (exchange, layout change, store).
template <typename R, int RA>
__device__ __forceinline__ void flush_neg(Regs<R, RA> &v, uint64_t &m)
{
    if (m) {
#pragma unroll
        for (int k = 0; k < RA; ++k)
            if ((m >> k) & 1) { v.setr(k, -v.getr(k)); v.seti(k, -v.geti(k)); }
        m = 0;
    }
}

template <int M, int RB, int VEC, typename R, int RA>
__device__ __forceinline__ void relayout(int from, int to, Regs<R, RA> &v, R *sm, int tid)
{
    __syncthreads();
    switch (from) {
    case 0: store_layout<M, RB, VEC, 0>(v, sm, tid); break;
    case 1: store_layout<M, RB, VEC, 1>(v, sm, tid); break;
    case 2: store_layout<M, RB, VEC, 2>(v, sm, tid); break;
    case 3: store_layout<M, RB, VEC, 3>(v, sm, tid); break;
    default: break;
    }
    __syncthreads();
    switch (to) {
    case 0: load_layout<M, RB, VEC, 0>(v, sm, tid); break;
    case 1: load_layout<M, RB, VEC, 1>(v, sm, tid); break;
    case 2: load_layout<M, RB, VEC, 2>(v, sm, tid); break;
    case 3: load_layout<M, RB, VEC, 3>(v, sm, tid); break;
    default: break;
    }
}

// ops staged in shared memory per chunk: every field read of the op loop is
// then a broadcast shared load instead of a dependent global load
constexpr int kOpChunk = 64;
static_assert(sizeof(StOp<float>) % 16 == 0 && sizeof(StOp<double>) % 16 == 0, "ops are copied as 16-byte vectors");
template <typename R>
__host__ __device__ constexpr size_t op_stage_bytes() { return (size_t)kOpChunk * sizeof(StOp<R>); }

// Apply an encoded op list to the registers of one tile (the whole body of a
// pass between the global load and store).  base = global index bits of the
// tile outside Q; sm = the tile's shared memory (2^M amplitudes); sops =
// shared memory for kOpChunk ops.  Every thread of the CTA runs the same op
// sequence (the chunk copies are CTA-wide).
template <typename R, int M, bool kRamp = false>
__device__ __forceinline__ void apply_ops(Regs<R, (1 << (M - kThrBits))> &v, const StOp<R> *__restrict__ gops,
                                          int nops, uint64_t base, int tid, R *sm, StOp<R> *sops)
{
    constexpr int VEC = (sizeof(R) == 4) ? 2 : 1;
    constexpr int RB = M - kThrBits;
    constexpr int RA = 1 << RB;
    int layout = 0;
    uint64_t negm = 0;
    const StOp<R> *ops = sops;
    for (int p0 = 0; p0 < nops; p0 += kOpChunk) {
    const int cnt = min(kOpChunk, nops - p0);
    {
        // this chunk of ops into shared memory (after every thread is done with the last one)
        __syncthreads();
        const uint4 *src = reinterpret_cast<const uint4 *>(gops + p0);
        uint4 *dst = reinterpret_cast<uint4 *>(sops);
        constexpr int W = (int)(sizeof(StOp<R>) / 16);
        for (int e = tid; e < cnt * W; e += kThr) dst[e] = __ldg(src + e);
        __syncthreads();
    }
    for (int p = 0; p < cnt; ++p) {
        const int kind = ops[p].kind;
        const int arg = ops[p].arg;
        if (kind == SK_LAYOUT) {
            flush_neg(v, negm);
            relayout<M, RB, VEC>(layout, arg, v, sm, tid);
            layout = arg;
            continue;
        }
        if (kind == SK_NOP) continue;
        // passes with ramps run the kernel variant compiled with kRamp (the
        // ramp's code costs registers the other passes need)
        if (kRamp && kind == SK_RAMP) {
            // the records of one ramp never straddle a chunk (the planner pads)
            const StOp<R> *rp = ops + p;
            auto entry = [&](int e, R &fr, R &fi) {
                fr = rp[e >> 2].m[2 * (e & 3)];
                fi = rp[e >> 2].m[2 * (e & 3) + 1];
            };
            const bool qt = ((tid & rp->thr_t) != 0) || ((base & rp->out_t) != 0);
            const uint64_t one = qt ? ~0ull : rp->km_t;
            if (one) {
                // the thread's factor from its low and high four thread bits
                R ar, ai, br, bi;
                entry(RA + (tid & 15), ar, ai);
                entry(RA + 16 + ((tid >> 4) & 15), br, bi);
                const R Fr = ar * br - ai * bi, Fi = ar * bi + ai * br;
#pragma unroll
                for (int k = 0; k < RA; ++k)
                    if ((one >> k) & 1) {
                        R gr, gi;
                        entry(k, gr, gi);
                        const R Gr = Fr * gr - Fi * gi, Gi = Fr * gi + Fi * gr;
                        const R vr = v.getr(k), vi = v.geti(k);
                        v.setr(k, Gr * vr - Gi * vi);
                        v.seti(k, Gr * vi + Gi * vr);
                    }
            }
            p += ramp_records(RA) - 1;
            continue;
        }
        const bool tok = ((tid & ops[p].thr_c) == ops[p].thr_c) && ((base & ops[p].out_c) == ops[p].out_c);
        CoefS<R> c;
        c.ar = ops[p].m[0]; c.ai = ops[p].m[1]; c.br = ops[p].m[2]; c.bi = ops[p].m[3];
        c.cr = ops[p].m[4]; c.ci = ops[p].m[5]; c.dr = ops[p].m[6]; c.di = ops[p].m[7];
        if (kind <= SK_XPERM) {
            flush_neg(v, negm);
            const bool plain = ops[p].plain != 0;
            const uint64_t act = tok ? ops[p].km_c : 0ull;
            if (kind == SK_DENSE) {
                if (plain) xdispatch<SK_DENSE, true>(arg, v, act, c);
                else xdispatch<SK_DENSE, false>(arg, v, act, c);
            } else if (kind == SK_ANTI) {
                if (plain) xdispatch<SK_ANTI, true>(arg, v, act, c);
                else xdispatch<SK_ANTI, false>(arg, v, act, c);
            } else {
                if (plain) xdispatch<SK_XPERM, true>(arg, v, act, c);
                else xdispatch<SK_XPERM, false>(arg, v, act, c);
            }
        } else {
            // diagonal: registers whose condition holds (km_c) and whose
            // target bit is 1 (km_t); the thread / tile part of the target
            // bit is ctb
            const bool ctb = ((tid & ops[p].thr_t) != 0) || ((base & ops[p].out_t) != 0);
            const uint64_t cond = tok ? ops[p].km_c : 0ull;
            const uint64_t one = ctb ? cond : (cond & ops[p].km_t);
            if (kind == SK_NEG) {
                negm ^= one;
            } else if (kind == SK_PHASE) {
#pragma unroll
                for (int k = 0; k < RA; ++k)
                    if ((one >> k) & 1) {
                        const R vr = v.getr(k), vi = v.geti(k);
                        v.setr(k, c.dr * vr - c.di * vi);
                        v.seti(k, c.dr * vi + c.di * vr);
                    }
            } else {
#pragma unroll
                for (int k = 0; k < RA; ++k)
                    if ((cond >> k) & 1) {
                        const bool tb = (one >> k) & 1;
                        const R fr = tb ? c.dr : c.ar, fi = tb ? c.di : c.ai;
                        const R vr = v.getr(k), vi = v.geti(k);
                        v.setr(k, fr * vr - fi * vi);
                        v.seti(k, fr * vi + fi * vr);
                    }
            }
        }
    }
    }
    flush_neg(v, negm);
}

// ---------------------------------------------------------------- host planner
struct Pass {
    std::vector<int> high;      // global qubits of local bits kLow .. M-1
    std::vector<int> members;   // gate indices (a valid order)
};

// Greedy passes: scan the remaining gates in order; a gate joins the pass if
// it commutes with every gate skipped before it and its non-diagonal qubits
// fit in Q (adding up to M - kLow high qubits).
std::vector<Pass> form_passes(const std::vector<SGate> &g, int n, int M)
{
    std::vector<Pass> passes;
    std::vector<char> done(g.size(), 0);
    const uint64_t low = (1ull << kLow) - 1ull;
    const int cap = M - kLow;
    size_t first = 0;
    while (first < g.size()) {
        Pass ps;
        uint64_t qmask = low;
        uint64_t bx = 0, bd = 0;      // qubits where skipped gates act non-diagonally / diagonally
        for (size_t i = first; i < g.size(); ++i) {
            if (done[i]) continue;
            const uint64_t x = g[i].xq(), d = g[i].dq();
            const bool free_of_skipped = ((x & (bx | bd)) == 0) && ((d & bx) == 0);
            bool ok = false;
            if (free_of_skipped) {
                const uint64_t add = x & ~qmask;
                if ((int)ps.high.size() + __builtin_popcountll(add) <= cap) {
                    ok = true;
                    for (int q = 0; q < n; ++q)
                        if ((add >> q) & 1) { ps.high.push_back(q); qmask |= 1ull << q; }
                }
            }
            if (ok) {
                ps.members.push_back((int)i);
                done[i] = 1;
            } else {
                bx |= x;
                bd |= d;
            }
        }
        // fill the tile with unused qubits (lowest first)
        for (int q = kLow; q < n && (int)ps.high.size() < cap; ++q)
            if (!((qmask >> q) & 1)) { ps.high.push_back(q); qmask |= 1ull << q; }
        passes.push_back(ps);
        while (first < g.size() && done[first]) ++first;
    }
    return passes;
}

// a controlled phase on two qubits (phase on |11>, not a sign flip, which
// the lazy sign mask handles for free): a candidate for a ramp
inline bool ramp_candidate(const SGate &g)
{
    return g.op == OP_DIAG_HI && __builtin_popcountll(g.ctrl) == 1 && !(g.m[6] == -1.0 && g.m[7] == 0.0);
}

template <typename R>
struct PlanBuilder {
    int n, M, RB, VEC;
    std::vector<StOp<R>> ops;
    std::vector<int> order;       // circuit index of each emitted gate op
    int layout_changes = 0;
    size_t pass_start = 0;        // first op of the pass being scheduled (chunks count from it)
    bool allow_ramps = true;      // merge runs of controlled phases into SK_RAMP ops
    size_t filler = 0;            // SK_NOP records (a ramp's table records and padding)

    int local_of(const Pass &ps, int q) const
    {
        if (q < kLow) return q;
        for (size_t i = 0; i < ps.high.size(); ++i)
            if (ps.high[i] == q) return kLow + (int)i;
        return -1;
    }
    int reg_of(int l, int b) const
    {
        for (int j = 0; j < RB; ++j)
            if (reg_local(M, RB, VEC, l, j) == b) return j;
        return -1;
    }
    int thr_of(int l, int b) const
    {
        for (int i = 0; i < kThrBits; ++i)
            if (thr_local(M, RB, VEC, l, i) == b) return i;
        return -1;
    }

    void emit_gate(const Pass &ps, const SGate &g, int layout)
    {
        StOp<R> o;
        memset(&o, 0, sizeof o);
        uint32_t reg_c = 0, reg_t = 0;
        for (int q = 0; q < n; ++q) {
            if (!((g.ctrl >> q) & 1)) continue;
            const int b = local_of(ps, q);
            if (b < 0) o.out_c |= 1ull << q;
            else if (reg_of(layout, b) >= 0) reg_c |= 1u << reg_of(layout, b);
            else o.thr_c |= 1u << thr_of(layout, b);
        }
        for (int k = 0; k < 8; ++k) o.m[k] = (R)g.m[k];
        const int bt = local_of(ps, g.target);
        if (g.op == OP_DIAG || g.op == OP_DIAG_HI) {
            if (bt < 0) o.out_t = 1ull << g.target;
            else if (reg_of(layout, bt) >= 0) reg_t = 1u << reg_of(layout, bt);
            else o.thr_t = 1u << thr_of(layout, bt);
            const bool neg = g.m[6] == -1.0 && g.m[7] == 0.0;
            o.kind = (g.op == OP_DIAG) ? SK_DIAG : (neg ? SK_NEG : SK_PHASE);
        } else {
            o.kind = (g.op == OP_DENSE) ? SK_DENSE : (g.op == OP_ANTIDIAG) ? SK_ANTI : SK_XPERM;
            o.arg = reg_of(layout, bt);
        }
        const int RA = 1 << RB;
        for (int k = 0; k < RA; ++k) {
            if (((uint32_t)k & reg_c) == reg_c) o.km_c |= 1ull << k;
            if ((uint32_t)k & reg_t) o.km_t |= 1ull << k;
        }
        o.plain = (reg_c == 0 && o.thr_c == 0 && o.out_c == 0) ? 1 : 0;
        ops.push_back(o);
    }

    // one SK_RAMP: amplitudes with qubit q at 1 times the product of the phases
    // of the pairs (q, m) whose local qubit m is 1 (see SK_RAMP)
    void emit_ramp(const Pass &ps, int q, const std::vector<std::pair<int, const SGate *>> &pairs, int layout)
    {
        // the records stay inside one chunk of kOpChunk ops
        const int RA = 1 << RB, nrec = ramp_records(RA);
        while ((ops.size() - pass_start) % kOpChunk > (size_t)(kOpChunk - nrec)) {
            StOp<R> nop;
            memset(&nop, 0, sizeof nop);
            nop.kind = SK_NOP;
            ops.push_back(nop);
            ++filler;
        }
        // per-bit factors: register bit j, thread bit i (products of repeated pairs)
        std::complex<double> freg[8], fthr[kThrBits];
        for (auto &f : freg) f = 1.0;
        for (auto &f : fthr) f = 1.0;
        for (const auto &pm : pairs) {
            const int b = local_of(ps, pm.first);
            const int j = reg_of(layout, b);
            const std::complex<double> ph(pm.second->m[6], pm.second->m[7]);
            if (j >= 0) freg[j] *= ph;
            else fthr[thr_of(layout, b)] *= ph;
        }
        // the tables (see SK_RAMP), each entry one FP64 product rounded once
        std::vector<std::complex<double>> tab(4 * nrec, 1.0);
        for (int k = 0; k < RA; ++k)
            for (int j = 0; j < RB; ++j)
                if ((k >> j) & 1) tab[k] *= freg[j];
        for (int x = 0; x < 16; ++x)
            for (int i = 0; i < 4; ++i)
                if ((x >> i) & 1) {
                    tab[RA + x] *= fthr[i];
                    tab[RA + 16 + x] *= fthr[4 + i];
                }
        std::vector<StOp<R>> rec(nrec);
        memset(rec.data(), 0, sizeof(StOp<R>) * nrec);
        rec[0].kind = SK_RAMP;
        const int bq = local_of(ps, q);
        uint32_t reg_t = 0;
        if (bq < 0) rec[0].out_t = 1ull << q;
        else if (reg_of(layout, bq) >= 0) reg_t = 1u << reg_of(layout, bq);
        else rec[0].thr_t = 1u << thr_of(layout, bq);
        for (int k = 0; k < RA; ++k)
            if ((uint32_t)k & reg_t) rec[0].km_t |= 1ull << k;
        for (int e = 0; e < 4 * nrec; ++e) {
            rec[e >> 2].m[2 * (e & 3)] = (R)tab[e].real();
            rec[e >> 2].m[2 * (e & 3) + 1] = (R)tab[e].imag();
        }
        for (int r = 1; r < nrec; ++r) rec[r].kind = SK_NOP;
        filler += (size_t)(nrec - 1);
        for (int r = 0; r < nrec; ++r) ops.push_back(rec[r]);
    }

    void emit_layout(int l)
    {
        ++layout_changes;
        StOp<R> o;
        memset(&o, 0, sizeof o);
        o.kind = SK_LAYOUT;
        o.arg = l;
        ops.push_back(o);
    }

    // order the pass's gates (respecting non-commuting pairs) so that
    // consecutive exchange gates share a layout; returns the op count
    int schedule(const Pass &ps, const std::vector<SGate> &g)
    {
        const size_t P = ps.members.size();
        const size_t start = ops.size();
        pass_start = start;
        std::vector<int> indeg(P, 0);
        std::vector<std::vector<int>> succ(P);
        for (size_t a = 0; a < P; ++a)
            for (size_t b = a + 1; b < P; ++b)
                if (!commute(g[ps.members[a]], g[ps.members[b]])) {
                    succ[a].push_back((int)b);
                    indeg[b]++;
                }
        std::vector<char> emitted(P, 0);
        const int NL = n_layouts(M, RB);
        int layout = 0;
        size_t left = P;
        auto fits = [&](int i, int l) {
            const SGate &s = g[ps.members[i]];
            if (!s.xq()) return true;
            return reg_of(l, local_of(ps, s.target)) >= 0;
        };
        while (left) {
            // controlled phases wait while any other gate can run: the gates
            // that run first free more phases to join one ramp
            int pick = -1;
            for (size_t i = 0; i < P && pick < 0 && allow_ramps; ++i)
                if (!emitted[i] && indeg[i] == 0 && !ramp_candidate(g[ps.members[i]]) && fits((int)i, layout))
                    pick = (int)i;
            for (size_t i = 0; i < P && pick < 0; ++i)
                if (!emitted[i] && indeg[i] == 0 && fits((int)i, layout)) pick = (int)i;
            if (pick < 0) {
                int best = -1, bestc = -1;
                for (int l = 0; l < NL; ++l) {
                    if (l == layout) continue;
                    int c = 0;
                    for (size_t i = 0; i < P; ++i)
                        if (!emitted[i] && indeg[i] == 0 && fits((int)i, l)) ++c;
                    if (c > bestc) { bestc = c; best = l; }
                }
                emit_layout(best);
                layout = best;
                continue;
            }
            auto mark = [&](int i) {
                order.push_back(g[ps.members[i]].orig);
                emitted[i] = 1;
                --left;
                for (int s2 : succ[i]) indeg[s2]--;
            };
            if (allow_ramps && ramp_candidate(g[ps.members[pick]])) {
                // every controlled phase that could run now and shares a qubit
                // with this one goes into one ramp over the qubit they share
                // most (the partner qubit must be inside the tile)
                const SGate &a = g[ps.members[pick]];
                const int qa = a.target, qb = __builtin_ctzll(a.ctrl);
                auto partner = [&](const SGate &c, int q) {
                    const int t = c.target, u = __builtin_ctzll(c.ctrl);
                    return t == q ? u : (u == q ? t : -1);
                };
                std::vector<int> cand;
                for (size_t i = 0; i < P; ++i)
                    if (!emitted[i] && indeg[i] == 0 && ramp_candidate(g[ps.members[i]])) cand.push_back((int)i);
                int best_q = -1;
                size_t best = 0;
                for (int q : {qa, qb}) {
                    size_t c = 0;
                    for (int i : cand) {
                        const int m = partner(g[ps.members[i]], q);
                        if (m >= 0 && local_of(ps, m) >= 0) ++c;
                    }
                    if (c > best) { best = c; best_q = q; }
                }
                if (best >= 3) {
                    std::vector<std::pair<int, const SGate *>> pairs;
                    std::vector<int> used;
                    for (int i : cand) {
                        const int m = partner(g[ps.members[i]], best_q);
                        if (m >= 0 && local_of(ps, m) >= 0) {
                            pairs.push_back({m, &g[ps.members[i]]});
                            used.push_back(i);
                        }
                    }
                    emit_ramp(ps, best_q, pairs, layout);
                    for (int i : used) mark(i);
                    continue;
                }
            }
            emit_gate(ps, g[ps.members[pick]], layout);
            mark(pick);
        }
        if (layout != 0) emit_layout(0);
        return (int)(ops.size() - start);
    }
};

}  // namespace
}  // namespace qsim
