// fused.cu -- gates fused into k-qubit unitaries, built in FP64 on the GPU and
// applied to the state as a real GEMM on the tcgen05 tensor cores.
//
// The full-operator view of §1.3.2 (U_t = I (x) ... (x) U (x) ... (x) I) is
// exact but needs a 2^n x 2^n matrix; restricted to a block of k qubits it is
// a 2^k x 2^k unitary U_blk = G_m ... G_1 of the block's gates.  With the
// block qubits as the fast index, the state is a matrix X [rows x 2^k] and the
// block applies out = X U_blk^T: a GEMM.  Storing each row interleaved
// (re, im) makes it a real GEMM with K = N = 2^(k+1):
//     D[r, 2i+b] = sum_{j,a} X[r, 2j+a] * W[2j+a, 2i+b],
//     W[2j, 2i] = W[2j+1, 2i+1] = Re U_ij,  W[2j+1, 2i] = -Im U_ij,  W[2j, 2i+1] = Im U_ij,
// so the complex64 state is read and written in place, without de-interleaving.
//
// Precision: kind::tf32 keeps 10 mantissa bits, too few for an infidelity of
// 1e-6 over ~100 blocks.  Both operands are split x = x_hi + x_lo with x_hi
// = x rounded to TF32 and x_lo = (x - x_hi) rounded to TF32 (both to nearest,
// so the split carries no bias), and D = A_hi B_hi + A_hi B_lo + A_lo B_hi is
// accumulated in FP32 in tensor memory (3xTF32; Ootomo & Yokota 2022).  k = 6
// splits into FP16 parts of power-of-two-scaled operands instead (the same 22
// significant bits at twice the tensor rate; see k_fused_tmem6).  U_blk
// itself is formed in FP64 (k_fuse_build) before the split.
//
// Apply kernels: persistent, warp-specialised CTAs stream tiles of 128 rows
// (MMA M = 128) through shared memory with bulk copies; converter warps split
// each row into A_hi / A_lo (k <= 5: shared memory, canonical no-swizzle
// K-major layout of 8-row x 16-byte core matrices; k = 6: tensor memory), one
// thread issues the MMAs against W in shared memory, commits arrive on
// mbarriers, and consumer warps read the accumulator back (tcgen05.ld 32x32b)
// and write the rows to HBM.  Every wait is bounded; on a timeout the kernel
// records SIM_ETIMEOUT in a device status word, frees its tensor memory and
// returns.
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace qsim {

namespace {

constexpr int kRows = 128;              // MMA M, rows per CTA

struct FGate {                          // one gate of a block, in block-local qubits
    int32_t target;
    uint32_t ctrl;
    double m[8];
};
// A 4 x 4 matrix S on local qubits la < lb (a density matrix's channel) takes
// four consecutive records: the first has target kSuperHead and ctrl =
// la | lb << 8, then kSuperRow; record l holds row l of S (l = 2 (bit lb) +
// (bit la)) as four (re, im) pairs.
constexpr int32_t kSuperHead = -1, kSuperRow = -2;


// x rounded to TF32 (10 explicit mantissa bits), nearest with ties away from
// zero.  Both parts of a 3xTF32 split are rounded, not truncated: truncation
// (and the tensor core's own truncation of FP32 operands) shrinks every
// element by half a TF32 ulp on average, and that bias builds up as a drift
// of the norm over many blocks.
// (two integer operations: add half a TF32 ulp to the magnitude bits, then
// clear the 13 bits below the TF32 mantissa; a carry into the exponent is the
// correct rounding up to the next binade; states hold no inf / NaN)
__device__ __forceinline__ float tf32_rn(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}


// k = 6 runs on FP16 operands scaled by powers of two (see k_fused_tmem6):
// the state by 2^se, se from a bound on its norm, each block's W by 2^we, we
// from a host bound on the block's entries (kF16WExp for a unitary block).
constexpr int kF16WExp = 14;
constexpr int kF16WExpMin = -100, kF16WExpMax = 126;

// ------------------------------------------------------------------ FP64 builder
// U = G_m ... G_1 applied to the identity column by column in FP64 (the
// columns are 2^k-amplitude states of the block's qubits and evolve
// independently), then W (the real form) split into TF32 hi / lo in the
// B-operand layout: [hi | lo], each K x K, K-major.  k = 6: 2^we W split into
// FP16 hi / lo (both rounded to nearest) in the 16-bit layout, [hi | lo] again,
// we = wexp[block].
// Each block's columns are spread over kBuildSplit<KQ> CTAs of 8 columns
// (this GPU's FP64 pipe is narrow: one CTA per block left the build
// FP64-bound on a handful of SMs); CTA (block, part) writes the W entries of
// its input columns, kk in [2 c0, 2 c0 + 2 DC), for every output n.
template <int KQ>
constexpr int kBuildSplit = (1 << KQ) >= 8 ? (1 << KQ) / 8 : 1;

template <int KQ>
__global__ void __launch_bounds__(256) k_fuse_build(const FGate *__restrict__ gates, const int *__restrict__ goff,
                                                    const int *__restrict__ wexp, float *__restrict__ bout)
{
    constexpr int D = 1 << KQ;
    constexpr int K = 2 * D;
    constexpr int CS = kBuildSplit<KQ>;
    constexpr int DC = D / CS;               // columns of this CTA
    extern __shared__ double2 U[];          // U[i * DC + c], row i, local column c
    const int blk = blockIdx.x / CS, c0 = (blockIdx.x % CS) * DC;
    for (int e = threadIdx.x; e < D * DC; e += 256) U[e] = make_double2((e / DC) == (e % DC) + c0 ? 1.0 : 0.0, 0.0);
    __syncthreads();
    for (int g = goff[blk]; g < goff[blk + 1]; ++g) {
        const int t = gates[g].target;
        const uint32_t cm = gates[g].ctrl;
        if (t == kSuperHead) {
            // 4 x 4 on local qubits (la, lb): y_l = sum_k S[l][k] x_k over the
            // four rows that differ only in those bits
            const int la = (int)(cm & 0xFFu), lb = (int)((cm >> 8) & 0xFFu);
            for (int e = threadIdx.x; e < DC * (D / 4); e += 256) {
                const int c = e / (D / 4);
                int i0 = e % (D / 4);
                i0 = ((i0 >> la) << (la + 1)) | (i0 & ((1 << la) - 1));
                i0 = ((i0 >> lb) << (lb + 1)) | (i0 & ((1 << lb) - 1));
                const int idx[4] = {i0, i0 | (1 << la), i0 | (1 << lb), i0 | (1 << la) | (1 << lb)};
                double2 x[4];
#pragma unroll
                for (int l = 0; l < 4; ++l) x[l] = U[idx[l] * DC + c];
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const double *r = gates[g + l].m;
                    double yr = 0.0, yi = 0.0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        yr += r[2 * k] * x[k].x - r[2 * k + 1] * x[k].y;
                        yi += r[2 * k] * x[k].y + r[2 * k + 1] * x[k].x;
                    }
                    U[idx[l] * DC + c] = make_double2(yr, yi);
                }
            }
            __syncthreads();
            g += 3;
            continue;
        }
        const double ar = gates[g].m[0], ai = gates[g].m[1], br = gates[g].m[2], bi = gates[g].m[3];
        const double cr = gates[g].m[4], ci = gates[g].m[5], dr = gates[g].m[6], di = gates[g].m[7];
        for (int e = threadIdx.x; e < DC * (D / 2); e += 256) {
            const int c = e / (D / 2), p = e % (D / 2);
            const int i0 = ((p >> t) << (t + 1)) | (p & ((1 << t) - 1));
            if (((uint32_t)i0 & cm) != cm) continue;
            const int i1 = i0 | (1 << t);
            const double2 a = U[i0 * DC + c], b = U[i1 * DC + c];
            U[i0 * DC + c] = make_double2(ar * a.x - ai * a.y + br * b.x - bi * b.y, ar * a.y + ai * a.x + br * b.y + bi * b.x);
            U[i1 * DC + c] = make_double2(cr * a.x - ci * a.y + dr * b.x - di * b.y, cr * a.y + ci * a.x + dr * b.y + di * b.x);
        }
        __syncthreads();
    }
    float *out = bout + (size_t)blk * 2 * K * K;
    for (int e = threadIdx.x; e < K * 2 * DC; e += 256) {
        const int n = e / (2 * DC), kk = 2 * c0 + e % (2 * DC);   // B_store[n][kk] = W[kk][n]
        const int i = n >> 1, b = n & 1, j = kk >> 1, a = kk & 1;
        const double2 u = U[i * DC + (j - c0)];
        const double w = (a == b) ? u.x : (a == 1 ? -u.y : u.y);
        if constexpr (KQ == 6) {
            __half *o16 = reinterpret_cast<__half *>(out);
            const double ws = ldexp(w, wexp[blk]);
            const __half hi = __double2half(ws);
            const __half lo = __double2half(ws - (double)__half2float(hi));
            const uint32_t off = kmajor16_off(n, kk, K) >> 1;
            o16[off] = hi;
            o16[K * K + off] = lo;
        } else {
            const float hi = tf32_rn((float)w);
            const float lo = tf32_rn((float)(w - (double)hi));
            const uint32_t off = kmajor_off(n, kk, K) >> 2;
            out[off] = hi;
            out[K * K + off] = lo;
        }
    }
}

// ------------------------------------------------------------------ apply
struct ApplyArgs {
    int nq;             // qubits of the block (KQ)
    int pos[8];         // global qubits of the block, ascending (local bit i <-> pos[i])
    uint64_t rows;      // 2^(n - KQ)
    // k = 6 only: W was scaled by 2^wexp before its FP16 split; the state's
    // norm^2 at the start of the call is *nrm2 (device), and growth bounds
    // how much the blocks and gates launched since then can have raised it
    int wexp;
    const double *nrm2;
    double growth;
};

// ------------------------------------------------------------------ streamed apply (k <= 5)
// A tile is 128 rows x 2^k amplitudes: the 2^(k+7) amplitudes that share
// every index bit outside T = (block qubits) u (the 7 lowest other qubits).
// Bits 0 .. L-1 of the index all lie in T (L >= 7), so a tile is
// 2^(k+7-L) <= 32 contiguous runs of 2^L amplitudes (>= 1 KB each).
//   warp 9: streams tiles into a ring of S shared-memory stages, lane j
//       issuing the cp.async.bulk of run j; the stage's mbarrier counts the
//       bytes landed;
//   warps 0-3: thread r takes row r of a landed stage, frees the stage, and
//       writes the row's TF32 hi / lo parts (K-major core-matrix layout) into
//       one of AB A buffers once the MMAs that last read that buffer are done;
//   warp 8 (one thread): per K-step one MMA A_hi x [W_hi | W_lo] (N = 2K) and
//       one A_lo x W_hi (N = K) into one of two TMEM accumulators, so that
//       columns [0, K) hold A_hi W_hi + A_lo W_hi and [K, 2K) hold A_hi W_lo;
//       commit to that accumulator's mbarrier;
//   warps 4-7: drain the other accumulator (both halves, summed) to HBM.
// W (hi / lo) is loaded once per CTA.  Every wait is bounded by %globaltimer;
// on a timeout the CTA records SIM_ETIMEOUT, lets copies and MMAs in flight
// land (bounded again), frees its tensor memory and returns.
constexpr int kStreamThreads = 320;


// S: stages in the ring; AB: A buffers (1 or 2); MINB: CTAs per SM the
// registers are budgeted for
template <int KQ> struct StreamCfg;
template <> struct StreamCfg<3> { static constexpr int S = 3, AB = 2, MINB = 2; };
template <> struct StreamCfg<4> { static constexpr int S = 2, AB = 2, MINB = 2; };
template <> struct StreamCfg<5> { static constexpr int S = 2, AB = 2, MINB = 1; };

template <int KQ>
__global__ void __launch_bounds__(kStreamThreads, StreamCfg<KQ>::MINB)
    k_fused_stream(float *__restrict__ st, const float *__restrict__ bmat, ApplyArgs a, uint64_t ntiles,
                   int *__restrict__ status)
{
    constexpr int S = StreamCfg<KQ>::S;
    constexpr int AB = StreamCfg<KQ>::AB;
    static_assert(AB == 1 || AB == 2, "one or two A buffers");
    constexpr int D = 1 << KQ;
    constexpr int K = 2 * D;
    constexpr int N = K;
    static_assert(4 * N <= 256, "two accumulators of 2N columns in half of tensor memory");
    constexpr int TB = KQ + 7;                       // tile bits
    constexpr int TAMP = 1 << TB;                    // amplitudes per tile = kRows * D
    constexpr uint32_t TBYTES = (uint32_t)TAMP * 8u;
    constexpr uint32_t NC = 2 * N;                   // TMEM columns per accumulator: [hi part | lo part]
    constexpr uint32_t NCOLS = 2 * NC;
    static_assert(NCOLS >= 32 && (NCOLS & (NCOLS - 1)) == 0, "TMEM allocations are powers of two >= 32");
    constexpr uint32_t SBO = (K / 4) * 128;
    constexpr uint32_t IDESC2 = make_idesc_tf32(kRows, 2 * N);
    constexpr uint32_t IDESC1 = make_idesc_tf32(kRows, N);
    constexpr int ABUF = kRows * K;                  // floats of one A operand

    extern __shared__ __align__(1024) unsigned char smem[];
    float2 *stage = reinterpret_cast<float2 *>(smem);                           // S x TAMP amplitudes
    float *abuf = reinterpret_cast<float *>(smem + (size_t)S * TBYTES);         // [buffer][hi | lo] kRows x K
    float *b_hi = abuf + 2 * AB * ABUF;                                          // N x K, then b_lo (N x K)
    __shared__ uint64_t bar_full[S], bar_empty[S], bar_a[2], bar_d[2], bar_e[2];
    __shared__ uint32_t tslot;
    __shared__ int tpos[TB];          // global bit of tile-local bit j (ascending)
    __shared__ uint64_t pmask;        // block bits
    __shared__ int lrun;              // L: tile-local bits 0 .. L-1 are global bits 0 .. L-1
    __shared__ uint32_t uc[D];        // tile-local offset of column c
    __shared__ uint64_t gc[D];        // global offset of column c
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        failed = *reinterpret_cast<volatile int *>(status);
        uint64_t pm = 0;
        for (int i = 0; i < KQ; ++i) pm |= 1ull << a.pos[i];
        uint64_t tm = pm;
        for (int b = 0, cnt = 0; cnt < 7; ++b)
            if (!((pm >> b) & 1)) { tm |= 1ull << b; ++cnt; }
        for (int b = 0, j = 0; j < TB; ++b)
            if ((tm >> b) & 1) tpos[j++] = b;
        int L = 0;
        while (L < TB && tpos[L] == L) ++L;
        lrun = L;
        pmask = pm;
    }
    __syncthreads();
    if (failed) return;
    if (warp == 0) tmem_alloc(&tslot, NCOLS);
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_empty[s], kRows);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar_a[b], kRows);
            mbar_init(&bar_d[b], 1);
            mbar_init(&bar_e[b], kRows);
        }
    }
    for (int c = tid; c < D; c += kStreamThreads) {
        uint32_t u = 0;
        uint64_t g = 0;
        for (int i = 0; i < KQ; ++i)
            if ((c >> i) & 1) {
                g |= 1ull << a.pos[i];
                for (int j = 0; j < TB; ++j)
                    if (tpos[j] == a.pos[i]) u |= 1u << j;
            }
        uc[c] = u;
        gc[c] = g;
    }
    {
        const float4 *src = reinterpret_cast<const float4 *>(bmat);
        float4 *dst = reinterpret_cast<float4 *>(b_hi);
        for (int e = tid; e < 2 * N * K / 4; e += kStreamThreads) dst[e] = __ldg(src + e);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tslot;
    volatile int *vfailed = &failed;
    const uint64_t step = gridDim.x;
    const int iters = ((uint64_t)blockIdx.x < ntiles) ? (int)((ntiles - 1 - blockIdx.x) / step + 1) : 0;

    // global index of tile t's first amplitude: zero bits inserted at T
    auto tile_base = [&](uint64_t t) {
        uint64_t b = t;
#pragma unroll
        for (int j = 0; j < TB; ++j) {
            const int p = tpos[j];
            b = ((b >> p) << (p + 1)) | (b & ((1ull << p) - 1ull));
        }
        return b;
    };
    // row r: its tile-local offset and global offset (row bits = T minus the block bits)
    auto row_offsets = [&](int r, uint32_t &u, uint64_t &g) {
        u = 0;
        g = 0;
        const uint64_t pm = pmask;
        for (int j = 0, i = 0; j < TB; ++j) {
            const int p = tpos[j];
            if ((pm >> p) & 1) continue;
            if ((r >> i) & 1) {
                u |= 1u << j;
                g |= 1ull << p;
            }
            ++i;
        }
    };

    if (warp == 9) {
        // loader warp: lane j copies run j of every tile
        const int L = lrun;
        const int nrun = 1 << (TB - L);
        const uint32_t rbytes = 8u << L;
        uint64_t go = 0;
        for (int b = 0; b < TB - L; ++b)
            if ((lane >> b) & 1) go |= 1ull << tpos[L + b];
        int issued = 0;
        for (int i = 0; i < iters && !warp_flag(vfailed); ++i) {
            const int s = i % S;
            if (i >= S && !mbar_wait_warp(&bar_empty[s], (uint32_t)((i / S - 1) & 1))) {
                *vfailed = 1;
                break;
            }
            const uint64_t base = tile_base(blockIdx.x + (uint64_t)i * step);
            if (lane == 0) mbar_arrive_expect_tx(&bar_full[s], TBYTES);
            __syncwarp();
            if (lane < nrun)
                bulk_load(stage + (size_t)s * TAMP + ((size_t)lane << L), st + 2 * (base | go), rbytes, &bar_full[s]);
            issued = i + 1;
        }
        // copies still in flight land before the CTA may exit
        if (lane == 0)
            for (int i = (issued > S ? issued - S : 0); i < issued; ++i)
                mbar_wait_bounded(&bar_full[i % S], (uint32_t)((i / S) & 1));
    } else if (warp < 4) {
        uint32_t ur;
        uint64_t gr;
        row_offsets(tid, ur, gr);
        // Bank spreading: with zc block bits among tile-local bits 0..3, the
        // 16 threads of a half-warp differ in their row's zr = 4 - zc low
        // tile bits only, so thread r reads column c ^ x with
        // x = (r >> zr) mod 2^zc: the low 4 tile-local bits (one 8-byte word
        // per bank pair) are then distinct across the half-warp.  uc is
        // linear over XOR, so column c ^ x sits at (ur | uc[c]) ^ uc[x].
        int zc = 0;
        for (int j = 0; j < 4; ++j) zc += (int)((pmask >> tpos[j]) & 1);
        const int x = (tid >> (4 - zc)) & ((1 << zc) - 1);
        const uint32_t ux = uc[x];
        for (int i = 0; i < iters && !warp_flag(vfailed); ++i) {
            const int s = i % S;
            if (!mbar_wait_warp(&bar_full[s], (uint32_t)((i / S) & 1))) {
                *vfailed = 1;
                break;
            }
            const float2 *sg = stage + (size_t)s * TAMP;
            float2 v[D];            // v[j] = column j ^ x of row tid
#pragma unroll
            for (int j = 0; j < D; ++j) v[j] = sg[(ur | uc[j]) ^ ux];
            mbar_arrive(&bar_empty[s]);
            // A buffer i % AB: the MMAs of tile i - AB must be done reading it
            if (i >= AB && !mbar_wait_warp(&bar_d[(i - AB) & 1], (uint32_t)(((i - AB) >> 1) & 1))) {
                *vfailed = 1;
                break;
            }
            unsigned char *ahi = reinterpret_cast<unsigned char *>(abuf + (size_t)(i % AB) * 2 * ABUF);
            unsigned char *alo = ahi + ABUF * sizeof(float);
#pragma unroll
            for (int j = 0; j < D; j += 2) {
                // columns 2p, 2p + 1 (p = (j ^ x) / 2) = one 16-byte row chunk
                // of a core matrix; x odd swaps which register holds which
                const uint32_t off = kmajor_off(tid, 2 * ((j ^ x) & ~1), K);
                const float2 e0 = (x & 1) ? v[j + 1] : v[j], e1 = (x & 1) ? v[j] : v[j + 1];
                const float h0 = tf32_rn(e0.x), h1 = tf32_rn(e0.y);
                const float h2 = tf32_rn(e1.x), h3 = tf32_rn(e1.y);
                *reinterpret_cast<float4 *>(ahi + off) = make_float4(h0, h1, h2, h3);
                *reinterpret_cast<float4 *>(alo + off) = make_float4(tf32_rn(e0.x - h0), tf32_rn(e0.y - h1),
                                                                     tf32_rn(e1.x - h2), tf32_rn(e1.y - h3));
            }
            fence_async_smem();
            mbar_arrive(&bar_a[i % AB]);
        }
    } else if (warp < 8) {
        // consumers: warp w reads TMEM lanes 32 (w - 4) .. + 31 = rows of the tile
        const int r = tid - 128;
        uint32_t ur;
        uint64_t gr;
        row_offsets(r, ur, gr);
        const bool q0_in_block = (pmask & 1ull) != 0;
        for (int i = 0; i < iters && !warp_flag(vfailed); ++i) {
            const int sb = i & 1;
            const uint64_t base = tile_base(blockIdx.x + (uint64_t)i * step) | gr;
            if (!mbar_wait_warp(&bar_d[sb], (uint32_t)((i >> 1) & 1))) {
                *vfailed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t lane_base = taddr + (uint32_t)(sb * NC) + ((uint32_t)((warp - 4) * 32) << 16);
            constexpr int W = N < 32 ? N : 32;            // columns per round (16 complex at most)
#pragma unroll
            for (int col = 0; col < N; col += W) {
                uint32_t hi[W], lo[W];
                if constexpr (W == 32) {
                    tmem_ld32_nowait(lane_base + (uint32_t)col, hi);
                    tmem_ld32_nowait(lane_base + (uint32_t)(N + col), lo);
                } else {
                    static_assert(W == 16, "N is 16, 32 or 64");
                    tmem_ld16_nowait(lane_base + (uint32_t)col, hi);
                    tmem_ld16_nowait(lane_base + (uint32_t)(N + col), lo);
                }
                tmem_wait_ld();
                float v[W];
#pragma unroll
                for (int e = 0; e < W; ++e) v[e] = __uint_as_float(hi[e]) + __uint_as_float(lo[e]);
                if (q0_in_block) {
                    // columns c, c + 1 are neighbouring amplitudes: one 16-byte store
#pragma unroll
                    for (int e = 0; e < W / 2; e += 2)
                        *reinterpret_cast<float4 *>(st + 2 * (base | gc[col / 2 + e])) =
                            make_float4(v[2 * e], v[2 * e + 1], v[2 * e + 2], v[2 * e + 3]);
                } else {
#pragma unroll
                    for (int e = 0; e < W / 2; ++e)
                        *reinterpret_cast<float2 *>(st + 2 * (base | gc[col / 2 + e])) =
                            make_float2(v[2 * e], v[2 * e + 1]);
                }
            }
            tc_fence_before();
            mbar_arrive(&bar_e[sb]);
        }
    } else if (lane == 0) {
        // issuer (warp 8, one thread)
        const uint32_t sb_hi = smem_u32(b_hi);
        for (int i = 0; i < iters && !*vfailed; ++i) {
            const int sb = i & 1;
            if (!mbar_wait_bounded(&bar_a[i % AB], (uint32_t)((i / AB) & 1))) { *vfailed = 1; break; }
            if (i >= 2 && !mbar_wait_bounded(&bar_e[sb], (uint32_t)(((i - 2) >> 1) & 1))) { *vfailed = 1; break; }
            tc_fence_after();
            const uint32_t sa_hi = smem_u32(abuf + (size_t)(i % AB) * 2 * ABUF), sa_lo = sa_hi + ABUF * sizeof(float);
            const uint32_t d = taddr + (uint32_t)(sb * NC);
#pragma unroll 1
            for (int ks = 0; ks < K / 8; ++ks) {
                const uint32_t ko = (uint32_t)ks * 256;
                // B rows 0 .. 2N-1 = W_hi then W_lo (contiguous, same 8-row group stride)
                mma_tf32(d, make_desc(sa_hi + ko, 128, SBO), make_desc(sb_hi + ko, 128, SBO), IDESC2, ks > 0);
                mma_tf32(d, make_desc(sa_lo + ko, 128, SBO), make_desc(sb_hi + ko, 128, SBO), IDESC1, 1);
            }
            mma_commit(&bar_d[sb]);
        }
    }
    if (*vfailed) {
        if (tid == 0) atomicExch(status, SIM_ETIMEOUT);
        // give tensor-core work still in flight a bounded chance to finish
        if (tid == 256 && iters > 0) mbar_wait_bounded(&bar_d[(iters - 1) & 1], (uint32_t)(((iters - 1) >> 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, NCOLS);
}

template <int KQ>
size_t stream_smem_bytes()
{
    constexpr int K = 2 << KQ;
    return (size_t)StreamCfg<KQ>::S * ((size_t)kRows << KQ) * 8 +
           (size_t)(2 * StreamCfg<KQ>::AB * kRows * K + 2 * K * K) * sizeof(float);
}

// ------------------------------------------------------------------ k = 6: FP16 split, A in tensor memory
// For k = 6 (K = N = 128) the tensor work per amplitude doubles and 3xTF32
// operands do not fit next to a stage ring (W hi | lo alone is 128 KB), so
// this kernel splits into FP16 instead: x = x_hi + x_lo with both parts FP16
// rounded to nearest, after scaling the state and W by exact powers of two.
// An FP16 part carries 11 significant bits like a TF32 part, so hi + lo keeps
// 22 bits as in 3xTF32, and kind::f16 runs at twice the rate of kind::tf32.
// Scales.  FP16 has a 5-bit exponent, so the scales follow the data.  Every
// amplitude is at most the state's norm, and a block multiplies the norm by
// at most its spectral norm; so with B^2 = nrm2 x growth (the norm^2 measured
// at the start of the call times the bound on what the blocks and gates
// launched since then can have added), 2^E <= B < 2^(E+1) and se = 14 - E
// (clamped to [-126, 126]), every scaled component is below 2^15, so the FP16
// maximum (65504) is not reached even if rounding had raised the norm by
// almost a factor 2, and amplitudes down to 2^-17 B keep 22 significant bits
// whatever the state's magnitude; smaller ones keep an absolute error below
// 2^-39 B (an infidelity contribution below 2^-78 per amplitude).  A state
// whose norm^2 overflows FP64 or is not a number cannot occur for finite
// complex64 amplitudes.
// W is scaled by 2^we, we from a host bound on the block's entries (14 for a
// unitary block).  The product is linear, so D = 2^(se + we) x (state W) up to
// the split; the consumer multiplies by 2^-(se + we) (in two exact steps when
// that factor is not a normal float).
// D = A_lo W_hi + A_hi W_lo + A_hi W_hi is accumulated in FP32 in tensor
// memory, the two small products first over all K-steps: the tensor core's
// accumulation truncates, and adding the small products before the
// accumulator is large keeps their share of that bias negligible.
// Tensor memory: A buffers of 128 columns (FP16 pairs: A_hi in the first 64,
// A_lo in the next 64) at [0, 128) and [128, 256), accumulators at [256, 384)
// and [384, 512).  Shared memory: two 64 KB stages and W (hi | lo, 32 KB each).
// Roles (320 threads), tile i uses stage, A buffer and accumulator i mod 2:
//   warp 9: the stage <- tile i (bulk copies of the runs of T) once the
//       converters have read tile i - 2 out of it;
//   warps 0-3: row r of the stage -> registers -> scaled FP16 hi / lo ->
//       TMEM lane r of A buffer i mod 2, once the MMAs of tile i - 2 are done;
//   warp 8 (one thread): the 24 MMAs of tile i once A is written and the
//       accumulator has been drained (tile i - 2);
//   warps 4-7: accumulator -> 2^-(se + we) x -> HBM.
// Every wait is bounded as in k_fused_stream.
constexpr int kT6Threads = 320;


__global__ void __launch_bounds__(kT6Threads, 1)
    k_fused_tmem6(float *__restrict__ st, const __half *__restrict__ bmat, ApplyArgs a, uint64_t ntiles,
                  int *__restrict__ status)
{
    constexpr int KQ = 6;
    constexpr int D = 1 << KQ;
    constexpr int K = 2 * D;
    constexpr int TB = KQ + 7;                       // tile bits
    constexpr int TAMP = 1 << TB;                    // amplitudes per tile
    constexpr uint32_t TBYTES = (uint32_t)TAMP * 8u;
    constexpr uint32_t NCOLS = 512;
    constexpr uint32_t COL_A = 0, COL_D = 256;       // + 128 per buffer
    constexpr uint32_t SBO = (K / 8) * 128;          // 8-row group stride of W, bytes
    constexpr uint32_t WLO = (uint32_t)K * K * 2u;   // byte offset of W_lo
    constexpr uint32_t IDESC = make_idesc_f16(kRows, K);

    extern __shared__ __align__(1024) unsigned char smem[];
    float2 *stage = reinterpret_cast<float2 *>(smem);                    // 2 x TAMP amplitudes
    __half *wsm = reinterpret_cast<__half *>(smem + 2 * (size_t)TBYTES); // [hi | lo] K x K each
    __shared__ uint64_t bar_full[2], bar_empty[2], bar_a[2], bar_d[2], bar_e[2];
    __shared__ uint32_t tslot;
    __shared__ int tpos[TB];          // global bit of tile-local bit j (ascending)
    __shared__ uint64_t pmask;        // block bits
    __shared__ int lrun;              // L: tile-local bits 0 .. L-1 are global bits 0 .. L-1
    __shared__ uint32_t uc[D];        // tile-local offset of column c
    __shared__ uint64_t gc[D];        // global offset of column c
    __shared__ int failed, sexp;      // sexp: se, the state's scale exponent

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        failed = *reinterpret_cast<volatile int *>(status);
        // B^2 = nrm2 x growth; 2^e2 <= B^2 < 2^(e2 + 1) gives 2^E <= B < 2^(E + 1)
        // with E = floor(e2 / 2); se = 14 - E
        double b2 = *a.nrm2 * a.growth;
        if (!(b2 > 0.0)) b2 = 0.0;                                    // NaN or zero: any scale
        const int e2 = (int)((__double_as_longlong(b2) >> 52) & 0x7ff) - 1023;   // -1023 for 0 / subnormal
        sexp = max(-126, min(126, 14 - (e2 >> 1)));                    // E = floor(e2 / 2)
        uint64_t pm = 0;
        for (int i = 0; i < KQ; ++i) pm |= 1ull << a.pos[i];
        uint64_t tm = pm;
        for (int b = 0, cnt = 0; cnt < 7; ++b)
            if (!((pm >> b) & 1)) { tm |= 1ull << b; ++cnt; }
        for (int b = 0, j = 0; j < TB; ++b)
            if ((tm >> b) & 1) tpos[j++] = b;
        int L = 0;
        while (L < TB && tpos[L] == L) ++L;
        lrun = L;
        pmask = pm;
    }
    __syncthreads();
    if (failed) return;
    if (warp == 0) tmem_alloc(&tslot, NCOLS);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar_full[b], 1);
            mbar_init(&bar_empty[b], kRows);
            mbar_init(&bar_a[b], kRows);
            mbar_init(&bar_d[b], 1);
            mbar_init(&bar_e[b], kRows);
        }
    }
    for (int c = tid; c < D; c += kT6Threads) {
        uint32_t u = 0;
        uint64_t g = 0;
        for (int i = 0; i < KQ; ++i)
            if ((c >> i) & 1) {
                g |= 1ull << a.pos[i];
                for (int j = 0; j < TB; ++j)
                    if (tpos[j] == a.pos[i]) u |= 1u << j;
            }
        uc[c] = u;
        gc[c] = g;
    }
    {
        const float4 *src = reinterpret_cast<const float4 *>(bmat);
        float4 *dst = reinterpret_cast<float4 *>(wsm);
        for (int e = tid; e < 2 * K * K * 2 / 16; e += kT6Threads) dst[e] = __ldg(src + e);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tslot;
    volatile int *vfailed = &failed;
    const uint64_t step = gridDim.x;
    const int iters = ((uint64_t)blockIdx.x < ntiles) ? (int)((ntiles - 1 - blockIdx.x) / step + 1) : 0;

    auto tile_base = [&](uint64_t t) {
        uint64_t b = t;
#pragma unroll
        for (int j = 0; j < TB; ++j) {
            const int p = tpos[j];
            b = ((b >> p) << (p + 1)) | (b & ((1ull << p) - 1ull));
        }
        return b;
    };
    auto row_offsets = [&](int r, uint32_t &u, uint64_t &g) {
        u = 0;
        g = 0;
        const uint64_t pm = pmask;
        for (int j = 0, i = 0; j < TB; ++j) {
            const int p = tpos[j];
            if ((pm >> p) & 1) continue;
            if ((r >> i) & 1) {
                u |= 1u << j;
                g |= 1ull << p;
            }
            ++i;
        }
    };

    if (warp == 9) {
        // loader warp: lane j copies runs j, j + 32 of every tile (T holds
        // qubits 0..6, so L >= 7 and there are at most 2^(TB - 7) = 64 runs)
        const int L = lrun;
        const int nrun = 1 << (TB - L);
        const uint32_t rbytes = 8u << L;
        int issued = 0;
        for (int i = 0; i < iters && !warp_flag(vfailed); ++i) {
            const int s = i & 1;
            if (i >= 2 && !mbar_wait_warp(&bar_empty[s], (uint32_t)(((i - 2) >> 1) & 1))) {
                *vfailed = 1;
                break;
            }
            const uint64_t base = tile_base(blockIdx.x + (uint64_t)i * step);
            if (lane == 0) mbar_arrive_expect_tx(&bar_full[s], TBYTES);
            __syncwarp();
            for (int rr = lane; rr < nrun; rr += 32) {
                uint64_t go = 0;
                for (int b = 0; b < TB - L; ++b)
                    if ((rr >> b) & 1) go |= 1ull << tpos[L + b];
                bulk_load(stage + (size_t)s * TAMP + ((size_t)rr << L), st + 2 * (base | go), rbytes, &bar_full[s]);
            }
            issued = i + 1;
        }
        // copies still in flight land before the CTA may exit
        if (lane == 0)
            for (int i = (issued > 2 ? issued - 2 : 0); i < issued; ++i)
                mbar_wait_bounded(&bar_full[i & 1], (uint32_t)((i >> 1) & 1));
    } else if (warp < 4) {
        uint32_t ur;
        uint64_t gr;
        row_offsets(tid, ur, gr);
        // bank spreading as in k_fused_stream: thread r reads column c ^ x,
        // then puts its registers back in column order by conditional swaps
        // (x < 16, so a half row of 32 columns maps onto itself)
        int zc = 0;
        for (int j = 0; j < 4; ++j) zc += (int)((pmask >> tpos[j]) & 1);
        const int x = (tid >> (4 - zc)) & ((1 << zc) - 1);
        const uint32_t ux = uc[x];
        const uint32_t tl = taddr + ((uint32_t)(warp * 32) << 16);
        const float xs = __uint_as_float((uint32_t)(sexp + 127) << 23);   // 2^se
        for (int i = 0; i < iters && !warp_flag(vfailed); ++i) {
            const int s = i & 1, b = i & 1;
            if (!mbar_wait_warp(&bar_full[s], (uint32_t)((i >> 1) & 1))) {
                *vfailed = 1;
                break;
            }
            // A buffer b: the MMAs of tile i - 2 must be done reading it
            if (i >= 2 && !mbar_wait_warp(&bar_d[b], (uint32_t)(((i - 2) >> 1) & 1))) {
                *vfailed = 1;
                break;
            }
            tc_fence_after();
            const float2 *sg = stage + (size_t)s * TAMP;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float2 v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = sg[(ur | uc[32 * h + j]) ^ ux];
                if (h == 1) mbar_arrive(&bar_empty[s]);
                if (zc > 0) {
#pragma unroll
                    for (int bb = 0; bb < 4; ++bb) {
                        if (bb < zc) {
                            const bool f = (x >> bb) & 1;
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (!((j >> bb) & 1)) {
                                    const float2 t0 = v[j], t1 = v[j | (1 << bb)];
                                    v[j] = f ? t1 : t0;
                                    v[j | (1 << bb)] = f ? t0 : t1;
                                }
                        }
                    }
                }
                // complex column j = K-elements 2j (re), 2j + 1 (im) = one 32-bit TMEM column
                uint32_t rh[32], rl[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float xr = v[j].x * xs, xi = v[j].y * xs;
                    const __half2 hh = __floats2half2_rn(xr, xi);
                    const float2 hf = __half22float2(hh);
                    const __half2 hl = __floats2half2_rn(xr - hf.x, xi - hf.y);
                    rh[j] = *reinterpret_cast<const uint32_t *>(&hh);
                    rl[j] = *reinterpret_cast<const uint32_t *>(&hl);
                }
                const uint32_t ab = tl + COL_A + 128u * (uint32_t)b + 32u * (uint32_t)h;
                tmem_st32(ab, rh);
                tmem_st32(ab + 64u, rl);
                tmem_wait_st();
            }
            tc_fence_before();
            mbar_arrive(&bar_a[b]);
        }
    } else if (warp < 8) {
        // consumers: warp w reads TMEM lanes 32 (w - 4) .. + 31 = rows of the tile
        const int r = tid - 128;
        uint32_t ur;
        uint64_t gr;
        row_offsets(r, ur, gr);
        const bool q0_in_block = (pmask & 1ull) != 0;
        // 2^-(se + we) as f1 f2, f2 = 1 unless 2^-t is not a normal float
        // (t in [-226, 252])
        const int t = sexp + a.wexp;
        const int t1 = (t >= -126 && t <= 126) ? t : t / 2;
        const float f1 = __uint_as_float((uint32_t)(127 - t1) << 23);
        const float f2 = __uint_as_float((uint32_t)(127 - (t - t1)) << 23);
        const bool two_step = t1 != t;
        for (int i = 0; i < iters && !warp_flag(vfailed); ++i) {
            const int b = i & 1;
            const uint64_t base = tile_base(blockIdx.x + (uint64_t)i * step) | gr;
            if (!mbar_wait_warp(&bar_d[b], (uint32_t)((i >> 1) & 1))) {
                *vfailed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t lane_base = taddr + COL_D + 128u * (uint32_t)b + ((uint32_t)((warp - 4) * 32) << 16);
#pragma unroll
            for (int col = 0; col < K; col += 32) {
                uint32_t d[32];
                tmem_ld32_nowait(lane_base + (uint32_t)col, d);
                tmem_wait_ld();
                float v[32];
#pragma unroll
                for (int e = 0; e < 32; ++e) v[e] = __uint_as_float(d[e]) * f1;
                if (two_step) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) v[e] *= f2;
                }
                if (q0_in_block) {
#pragma unroll
                    for (int e = 0; e < 16; e += 2)
                        *reinterpret_cast<float4 *>(st + 2 * (base | gc[col / 2 + e])) =
                            make_float4(v[2 * e], v[2 * e + 1], v[2 * e + 2], v[2 * e + 3]);
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        *reinterpret_cast<float2 *>(st + 2 * (base | gc[col / 2 + e])) =
                            make_float2(v[2 * e], v[2 * e + 1]);
                }
            }
            tc_fence_before();
            mbar_arrive(&bar_e[b]);
        }
    } else if (warp == 8 && lane == 0) {
        // issuer (one thread): per tile 8 K-steps x (A_lo W_hi), then A_hi W_lo, then A_hi W_hi
        const uint32_t sw = smem_u32(wsm);
        int nd = 0;                   // commits issued
        for (int i = 0; i < iters && !*vfailed; ++i) {
            const int b = i & 1;
            if (!mbar_wait_bounded(&bar_a[b], (uint32_t)((i >> 1) & 1))) { *vfailed = 1; break; }
            if (i >= 2 && !mbar_wait_bounded(&bar_e[b], (uint32_t)(((i - 2) >> 1) & 1))) { *vfailed = 1; break; }
            tc_fence_after();
            const uint32_t d = taddr + COL_D + 128u * (uint32_t)b;
            const uint32_t ahi = taddr + COL_A + 128u * (uint32_t)b, alo = ahi + 64u;
#pragma unroll 1
            for (int pass = 0; pass < 3; ++pass) {
                const uint32_t ac = pass == 0 ? alo : ahi;
                const uint32_t bw = sw + (pass == 1 ? WLO : 0u);
#pragma unroll 1
                for (int ks = 0; ks < K / 16; ++ks)
                    mma_f16_ta(d, ac + 8u * (uint32_t)ks, make_desc(bw + (uint32_t)ks * 256u, 128, SBO), IDESC,
                               (pass | ks) != 0);
            }
            mma_commit(&bar_d[b]);
            nd = i + 1;
        }
        // tensor-core work still in flight finishes before tensor memory is freed
        if (*vfailed && nd > 0) mbar_wait_bounded(&bar_d[(nd - 1) & 1], (uint32_t)(((nd - 1) >> 1) & 1));
    }
    __syncthreads();
    if (tid == 0 && *vfailed) atomicExch(status, SIM_ETIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, NCOLS);
}

constexpr size_t tmem6_smem_bytes() { return 2 * ((size_t)kRows << 6) * 8 + (size_t)2 * 128 * 128 * sizeof(__half); }

// ------------------------------------------------------------------ multi-block passes (k = 5)
// Several consecutive blocks whose qubits fit one 12-qubit tile set T are
// applied to each tile while it stays in shared memory: one HBM read and one
// write for the whole run of blocks instead of one per block.  For block j the
// tile is viewed as 128 rows (the 7 qubits of T outside the block) x 32
// columns (the block's qubits); the tile is kept in T's own index order.
//   warps 9-10: load tiles into a ring of two stages with 16-byte cp.async
//       (T may be any 12 qubits that include qubit 0, so runs can be as short
//       as two amplitudes); each loader thread's arrival on the stage's
//       mbarrier fires when its copies have landed;
//   warps 0-3: per block, row r of the current view into A (hi / lo, one
//       buffer, after the MMAs of the previous step are done with it);
//   warp 8: the 3xTF32 MMAs of the step with that block's W;
//   warps 4-7: drain the accumulator -- back into the tile in shared memory
//       for every block but the last, to HBM for the last.
// Steps s = (tile, block) run in order; every wait is bounded.
constexpr int kMaxPass = 2;
constexpr int kMultiThreads = 352;

struct PassArgs {
    int m;                       // blocks in the pass, 2..kMaxPass
    int tpos[12];                // tile qubits, ascending (tpos[0] = 0)
    int pos[kMaxPass][5];        // qubits of block j, ascending, all in tpos
};

__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint64_t *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__global__ void __launch_bounds__(kMultiThreads, 1)
    k_fused_multi(float *__restrict__ st, const float *__restrict__ bmat, PassArgs a, uint64_t ntiles,
                  int *__restrict__ status)
{
    constexpr int KQ = 5;
    constexpr int D = 1 << KQ;
    constexpr int K = 2 * D;
    constexpr int N = K;
    constexpr int TB = 12;
    constexpr int TAMP = 1 << TB;
    constexpr uint32_t NC = 2 * N;
    constexpr uint32_t NCOLS = 2 * NC;
    constexpr uint32_t SBO = (K / 4) * 128;
    constexpr uint32_t IDESC2 = make_idesc_tf32(kRows, 2 * N);
    constexpr uint32_t IDESC1 = make_idesc_tf32(kRows, N);
    constexpr int ABUF = kRows * K;
    constexpr int WBLK = 2 * N * K;              // floats of one block's W (hi then lo)
    constexpr int kLoaders = 64;

    extern __shared__ __align__(1024) unsigned char smem[];
    float2 *stage = reinterpret_cast<float2 *>(smem);                               // 2 x TAMP
    float *a_hi = reinterpret_cast<float *>(smem + 2 * (size_t)TAMP * sizeof(float2));
    float *a_lo = a_hi + ABUF;
    float *wbuf = a_lo + ABUF;                                                        // m x WBLK
    __shared__ uint64_t bar_full[2], bar_empty[2], bar_a, bar_d[2], bar_e[2], bar_w;
    __shared__ uint32_t tslot;
    __shared__ int tpos[TB];
    __shared__ uint32_t uc[kMaxPass][D];         // tile-local offset of column c in view j
    __shared__ uint32_t urs[kMaxPass][kRows];    // tile-local offset of row r in view j
    __shared__ uint64_t gr_last[kRows];          // global offset of row r in the last view
    __shared__ uint64_t gc_last[D];              // global offset of column c in the last view
    __shared__ uint64_t dlo[64], dhi[64];        // global offsets of tile-local index bits 0-5 / 6-11
    __shared__ int xs[kMaxPass];                 // bank spreading: zc of view j
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = a.m;
    if (tid == 0) failed = *reinterpret_cast<volatile int *>(status);
    if (tid < TB) tpos[tid] = a.tpos[tid];
    __syncthreads();
    if (failed) return;
    if (warp == 0) tmem_alloc(&tslot, NCOLS);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar_full[b], kLoaders);
            mbar_init(&bar_empty[b], kRows);
            mbar_init(&bar_d[b], 1);
            mbar_init(&bar_e[b], kRows);
        }
        mbar_init(&bar_a, kRows);
        mbar_init(&bar_w, kRows);
    }
    // view tables
    auto local_of = [&](int q) {
        for (int t = 0; t < TB; ++t)
            if (tpos[t] == q) return t;
        return 0;
    };
    for (int e = tid; e < kMaxPass * D; e += kMultiThreads) {
        const int j = e / D, c = e % D;
        uint32_t u = 0;
        if (j < m)
            for (int i = 0; i < KQ; ++i)
                if ((c >> i) & 1) u |= 1u << local_of(a.pos[j][i]);
        uc[j][c] = u;
        if (j == m - 1) {
            uint64_t g = 0;
            for (int i = 0; i < KQ; ++i)
                if ((c >> i) & 1) g |= 1ull << a.pos[j][i];
            gc_last[c] = g;
        }
    }
    for (int e = tid; e < kMaxPass * kRows; e += kMultiThreads) {
        const int j = e / kRows, r = e % kRows;
        uint32_t u = 0;
        uint64_t g = 0;
        if (j < m) {
            uint32_t pm = 0;
            for (int i = 0; i < KQ; ++i) pm |= 1u << local_of(a.pos[j][i]);
            for (int t = 0, i = 0; t < TB; ++t) {
                if ((pm >> t) & 1) continue;
                if ((r >> i) & 1) {
                    u |= 1u << t;
                    g |= 1ull << tpos[t];
                }
                ++i;
            }
        }
        urs[j][r] = u;
        if (j == m - 1) gr_last[r] = g;
    }
    for (int e = tid; e < 128; e += kMultiThreads) {
        const int hi = e >> 6, v = e & 63;
        uint64_t g = 0;
        for (int b = 0; b < 6; ++b)
            if ((v >> b) & 1) g |= 1ull << tpos[6 * hi + b];
        (hi ? dhi : dlo)[v] = g;
    }
    if (tid < kMaxPass) {
        int zc = 0;
        if (tid < m)
            for (int t = 0; t < 4; ++t)
                for (int i = 0; i < KQ; ++i) zc += (a.pos[tid][i] == tpos[t]);
        xs[tid] = zc;
    }
    {
        const float4 *src = reinterpret_cast<const float4 *>(bmat);
        float4 *dst = reinterpret_cast<float4 *>(wbuf);
        for (int e = tid; e < m * WBLK / 4; e += kMultiThreads) dst[e] = __ldg(src + e);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tslot;
    volatile int *vfailed = &failed;
    const uint64_t step = gridDim.x;
    const int iters = ((uint64_t)blockIdx.x < ntiles) ? (int)((ntiles - 1 - blockIdx.x) / step + 1) : 0;
    auto tile_base = [&](uint64_t t) {
        uint64_t b = t;
#pragma unroll
        for (int q = 0; q < TB; ++q) {
            const int p = tpos[q];
            b = ((b >> p) << (p + 1)) | (b & ((1ull << p) - 1ull));
        }
        return b;
    };

    if (warp >= 9) {
        // loaders: thread lt copies 16-byte pairs of amplitudes u = 2 (lt + 64 k)
        const int lt = tid - 9 * 32;
        for (int i = 0; i < iters && !warp_flag(vfailed); ++i) {
            const int sg = i & 1;
            if (i >= 2 && !mbar_wait_warp(&bar_empty[sg], (uint32_t)(((i >> 1) - 1) & 1))) {
                *vfailed = 1;
                break;
            }
            const uint64_t base = tile_base(blockIdx.x + (uint64_t)i * step);
            float2 *dst = stage + (size_t)sg * TAMP;
#pragma unroll 4
            for (int k = 0; k < TAMP / 2 / kLoaders; ++k) {
                const uint32_t u = 2u * (uint32_t)(lt + kLoaders * k);
                const uint64_t g = base | dlo[u & 63] | dhi[u >> 6];
                cp_async16(dst + u, st + 2 * g);
            }
            cp_async_arrive(&bar_full[sg]);
        }
        cp_async_wait_all();
    } else if (warp < 4) {
        for (int i = 0; i < iters && !warp_flag(vfailed); ++i) {
            const int sg = i & 1;
            const float2 *X = stage + (size_t)sg * TAMP;
            for (int j = 0; j < m && !warp_flag(vfailed); ++j) {
                const int s = i * m + j;
                bool ok;
                if (j == 0) ok = mbar_wait_warp(&bar_full[sg], (uint32_t)((i >> 1) & 1));
                else ok = mbar_wait_warp(&bar_w, (uint32_t)((i * (m - 1) + j - 1) & 1));
                if (!ok) { *vfailed = 1; break; }
                const int zc = xs[j];
                const int x = (tid >> (4 - zc)) & ((1 << zc) - 1);
                const uint32_t ur = urs[j][tid], ux = uc[j][x];
                float2 v[D];
#pragma unroll
                for (int c = 0; c < D; ++c) v[c] = X[(ur | uc[j][c]) ^ ux];
                if (j == m - 1) mbar_arrive(&bar_empty[sg]);
                if (s >= 1 && !mbar_wait_warp(&bar_d[(s - 1) & 1], (uint32_t)(((s - 1) >> 1) & 1))) {
                    *vfailed = 1;
                    break;
                }
                unsigned char *ahi = reinterpret_cast<unsigned char *>(a_hi);
                unsigned char *alo = reinterpret_cast<unsigned char *>(a_lo);
#pragma unroll
                for (int c = 0; c < D; c += 2) {
                    const uint32_t off = kmajor_off(tid, 2 * ((c ^ x) & ~1), K);
                    const float2 e0 = (x & 1) ? v[c + 1] : v[c], e1 = (x & 1) ? v[c] : v[c + 1];
                    const float h0 = tf32_rn(e0.x), h1 = tf32_rn(e0.y);
                    const float h2 = tf32_rn(e1.x), h3 = tf32_rn(e1.y);
                    *reinterpret_cast<float4 *>(ahi + off) = make_float4(h0, h1, h2, h3);
                    *reinterpret_cast<float4 *>(alo + off) = make_float4(tf32_rn(e0.x - h0), tf32_rn(e0.y - h1),
                                                                         tf32_rn(e1.x - h2), tf32_rn(e1.y - h3));
                }
                fence_async_smem();
                mbar_arrive(&bar_a);
            }
        }
    } else if (warp < 8) {
        const int r = tid - 128;
        const uint64_t gr = gr_last[r];
        const bool q0_last = a.pos[m - 1][0] == 0;
        for (int i = 0; i < iters && !warp_flag(vfailed); ++i) {
            const int sg = i & 1;
            float2 *X = stage + (size_t)sg * TAMP;
            const uint64_t base = tile_base(blockIdx.x + (uint64_t)i * step) | gr;
            for (int j = 0; j < m && !warp_flag(vfailed); ++j) {
                const int s = i * m + j;
                const int sb = s & 1;
                if (!mbar_wait_warp(&bar_d[sb], (uint32_t)((s >> 1) & 1))) { *vfailed = 1; break; }
                tc_fence_after();
                const uint32_t lane_base = taddr + (uint32_t)(sb * NC) + ((uint32_t)((warp - 4) * 32) << 16);
                const bool last = j == m - 1;
                const uint32_t ur = urs[j][r];
#pragma unroll
                for (int col = 0; col < N; col += 32) {
                    uint32_t hi[32], lo[32];
                    tmem_ld32_nowait(lane_base + (uint32_t)col, hi);
                    tmem_ld32_nowait(lane_base + (uint32_t)(N + col), lo);
                    tmem_wait_ld();
                    float v[32];
#pragma unroll
                    for (int e = 0; e < 32; ++e) v[e] = __uint_as_float(hi[e]) + __uint_as_float(lo[e]);
                    if (!last) {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            X[ur | uc[j][col / 2 + e]] = make_float2(v[2 * e], v[2 * e + 1]);
                    } else if (q0_last) {
#pragma unroll
                        for (int e = 0; e < 16; e += 2)
                            *reinterpret_cast<float4 *>(st + 2 * (base | gc_last[col / 2 + e])) =
                                make_float4(v[2 * e], v[2 * e + 1], v[2 * e + 2], v[2 * e + 3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            *reinterpret_cast<float2 *>(st + 2 * (base | gc_last[col / 2 + e])) =
                                make_float2(v[2 * e], v[2 * e + 1]);
                    }
                }
                tc_fence_before();
                mbar_arrive(&bar_e[sb]);
                if (!last) mbar_arrive(&bar_w);
            }
        }
    } else if (lane == 0) {
        const uint32_t sa_hi = smem_u32(a_hi), sa_lo = smem_u32(a_lo);
        for (int i = 0; i < iters && !*vfailed; ++i)
            for (int j = 0; j < m && !*vfailed; ++j) {
                const int s = i * m + j;
                const int sb = s & 1;
                if (!mbar_wait_bounded(&bar_a, (uint32_t)(s & 1))) { *vfailed = 1; break; }
                if (s >= 2 && !mbar_wait_bounded(&bar_e[sb], (uint32_t)(((s - 2) >> 1) & 1))) { *vfailed = 1; break; }
                tc_fence_after();
                const uint32_t sb_hi = smem_u32(wbuf + (size_t)j * WBLK);
                const uint32_t d = taddr + (uint32_t)(sb * NC);
#pragma unroll 1
                for (int ks = 0; ks < K / 8; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 256;
                    mma_tf32(d, make_desc(sa_hi + ko, 128, SBO), make_desc(sb_hi + ko, 128, SBO), IDESC2, ks > 0);
                    mma_tf32(d, make_desc(sa_lo + ko, 128, SBO), make_desc(sb_hi + ko, 128, SBO), IDESC1, 1);
                }
                mma_commit(&bar_d[sb]);
            }
    }
    if (*vfailed) {
        if (tid == 0) atomicExch(status, SIM_ETIMEOUT);
        const int last = iters * m - 1;
        if (tid == 256 && last >= 0) mbar_wait_bounded(&bar_d[last & 1], (uint32_t)((last >> 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, NCOLS);
}

size_t multi_smem_bytes(int m)
{
    constexpr int K = 64;
    return 2 * (size_t)4096 * sizeof(float2) + (size_t)(2 * kRows * K) * sizeof(float) +
           (size_t)m * 2 * K * K * sizeof(float);
}

// ------------------------------------------------------------------ host planner
struct Block {
    uint64_t qmask;
    std::vector<int> members;
    bool wide = false;        // one gate on more than k qubits: applied by a per-gate launch
};

// Fixed-k blocks with a lookahead choice of qubits.  A block starts from the
// qubits of the first remaining gate and grows up to k qubits; each growth
// step adds the set of at most `depth` further qubits that lets the most of
// the next gates (a window of 256 not yet placed) join -- a gate joins if all
// its qubits are in the set and it commutes with every gate skipped before it
// (ties: the smaller set, then the earlier candidates).  Then every remaining
// gate that commutes with the gates skipped before it and lies on the block's
// qubits joins.  depth 1 adds one qubit at a time; depth 2 also weighs pairs
// (two qubits that only pay off together, such as the two ends of a CZ),
// depth 3 triples (split over the host threads).
// Blocks come out one at a time, so that a caller can launch the first ones
// while it plans the rest.
class BlockPlanner {
public:
    BlockPlanner(const std::vector<SGate> &g, int k, int n, int depth)
        : g_(g), k_(k), n_(n), depth_(depth), done_(g.size(), 0) {}

    void set_depth(int d) { depth_ = d; }

    bool next(Block *b)
    {
        while (first_ < g_.size() && done_[first_]) ++first_;
        if (first_ >= g_.size()) return false;
        *b = Block{0, {}};
        uint64_t S = g_[first_].xq() | g_[first_].dq();
        if (__builtin_popcountll(S) > k_) {
            // the first remaining gate alone spans more than k qubits
            b->qmask = S;
            b->members.push_back((int)first_);
            b->wide = true;
            done_[first_] = 1;
            return true;
        }
        load_window();
        while (__builtin_popcountll(S) < k_) {
            const int free = k_ - __builtin_popcountll(S);
            std::vector<int> cand;
            for (int q = 0; q < n_; ++q)
                if (!((S >> q) & 1) && ((touched_ >> q) & 1)) cand.push_back(q);
            // bounds pay for themselves only where pairs and triples are
            // searched (measured: depth 1 runs faster without them)
            const bool prune = depth_ >= 2 && free >= 2;
            if (prune) load_bounds(S, std::min(depth_, free));
            int best = absorb(S);
            uint64_t best_add = 0;
            // a candidate replaces the best only with a strictly larger count,
            // so one whose bound is not larger is skipped without changing the
            // outcome
            for (size_t i = 0; i < cand.size(); ++i) {
                if (prune && bound1(cand[i]) <= best) continue;
                const uint64_t a1 = 1ull << cand[i];
                const int c1 = absorb(S | a1);
                if (c1 > best) { best = c1; best_add = a1; }
            }
            if (depth_ >= 2 && free >= 2) {
                for (size_t i = 0; i < cand.size(); ++i)
                    for (size_t j = i + 1; j < cand.size(); ++j) {
                        if (bound2(cand[i], cand[j]) <= best) continue;
                        const uint64_t a2 = (1ull << cand[i]) | (1ull << cand[j]);
                        const int c2 = absorb(S | a2);
                        if (c2 > best) { best = c2; best_add = a2; }
                    }
            }
            if (depth_ >= 3 && free >= 3) {
                // triples, split by their first candidate over host threads;
                // each slice keeps its first best, the earliest slice wins ties.
                // A triple is skipped when its bound is not above both the
                // best before the triples and its slice's best: it could then
                // neither be its slice's first maximum nor win the merge.
                const size_t nc = cand.size();
                const int floor = best;
                std::vector<int> sbest(nc, -1);
                std::vector<uint64_t> sadd(nc, 0);
                parallel_for(nc, [&](size_t i) {
                    for (size_t j = i + 1; j < nc; ++j)
                        for (size_t l = j + 1; l < nc; ++l) {
                            if (bound3(cand[i], cand[j], cand[l]) <= std::max(floor, sbest[i])) continue;
                            const uint64_t a3 = (1ull << cand[i]) | (1ull << cand[j]) | (1ull << cand[l]);
                            const int c3 = absorb(S | a3);
                            if (c3 > sbest[i]) { sbest[i] = c3; sadd[i] = a3; }
                        }
                });
                for (size_t i = 0; i < nc; ++i)
                    if (sbest[i] > best) { best = sbest[i]; best_add = sadd[i]; }
            }
            if (!best_add) break;
            S |= best_add;
        }
        uint64_t bx = 0, bd = 0;
        for (size_t i = first_; i < g_.size(); ++i) {
            if (done_[i]) continue;
            const uint64_t x = g_[i].xq(), d = g_[i].dq();
            if (((x & (bx | bd)) == 0) && ((d & bx) == 0) && (((x | d) & ~S) == 0)) {
                b->qmask |= x | d;
                b->members.push_back((int)i);
                done_[i] = 1;
            } else {
                bx |= x;
                bd |= d;
            }
        }
        return true;
    }

private:
    static constexpr size_t kWindow = 256;

    // the next kWindow not-placed gates as (non-diagonal, diagonal) masks
    void load_window()
    {
        wx_.clear();
        wd_.clear();
        touched_ = 0;
        for (size_t i = first_; i < g_.size() && wx_.size() < kWindow; ++i) {
            if (done_[i]) continue;
            wx_.push_back(g_[i].xq());
            wd_.push_back(g_[i].dq());
            touched_ |= g_[i].xq() | g_[i].dq();
        }
    }

    // Upper bounds on absorb(S | a) for the candidate sets a of one growth
    // step: every window gate counted once, by its qubits outside S (at most
    // `depth` of them); absorb(S | a) counts a subset of the gates whose
    // outside qubits lie in a, so bound(a) >= absorb(S | a).
    void load_bounds(uint64_t S, int depth)
    {
        c0_ = 0;
        c1_.assign((size_t)n_, 0);
        c2_.assign(depth >= 2 ? (size_t)n_ * n_ : 0, 0);
        c3_.clear();
        for (size_t i = 0; i < wx_.size(); ++i) {
            const uint64_t r = (wx_[i] | wd_[i]) & ~S;
            const int pc = __builtin_popcountll(r);
            if (pc == 0) {
                ++c0_;
            } else if (pc == 1) {
                ++c1_[(size_t)__builtin_ctzll(r)];
            } else if (pc == 2 && depth >= 2) {
                const int a = __builtin_ctzll(r), b = __builtin_ctzll(r & (r - 1));
                ++c2_[(size_t)a * n_ + b];
            } else if (pc == 3 && depth >= 3) {
                c3_.push_back(r);
            }
        }
        std::sort(c3_.begin(), c3_.end());
    }
    int bound1(int a) const { return c0_ + c1_[(size_t)a]; }
    // a < b < c (candidates ascending)
    int bound2(int a, int b) const { return c0_ + c1_[(size_t)a] + c1_[(size_t)b] + c2_[(size_t)a * n_ + b]; }
    int bound3(int a, int b, int c) const
    {
        const uint64_t m = (1ull << a) | (1ull << b) | (1ull << c);
        const auto r = std::equal_range(c3_.begin(), c3_.end(), m);
        return bound2(a, b) + c1_[(size_t)c] + c2_[(size_t)a * n_ + c] + c2_[(size_t)b * n_ + c] +
               (int)(r.second - r.first);
    }

    // gates of the window that could join a block on qubit set S
    int absorb(uint64_t S) const
    {
        uint64_t bx = 0, bd = 0;
        int cnt = 0;
        for (size_t i = 0; i < wx_.size(); ++i) {
            const uint64_t x = wx_[i], d = wd_[i];
            if (((x & (bx | bd)) == 0) && ((d & bx) == 0) && (((x | d) & ~S) == 0)) {
                ++cnt;
            } else {
                bx |= x;
                bd |= d;
            }
        }
        return cnt;
    }

    const std::vector<SGate> &g_;
    int k_, n_, depth_;
    std::vector<char> done_;
    size_t first_ = 0;
    std::vector<uint64_t> wx_, wd_;
    uint64_t touched_ = 0;
    int c0_ = 0;                      // bounds of the current growth step (load_bounds)
    std::vector<int> c1_, c2_;
    std::vector<uint64_t> c3_;
};

// Multi-block passes (k = 5): consecutive pairs of blocks whose qubits, with
// qubit 0, fit one 12-qubit tile run as one pass; tileset[b] = the tile's
// qubits (padded with the lowest others) for the first block of a pair, 0
// otherwise; second[b] marks the pair's second block.
void pair_blocks(const std::vector<Block> &blocks, int n, bool on, std::vector<uint64_t> *tileset,
                 std::vector<char> *second)
{
    tileset->assign(blocks.size(), 0);
    second->assign(blocks.size(), 0);
    if (!on || n < 12) return;
    for (size_t bi = 0; bi + 1 < blocks.size(); ++bi) {
        if (blocks[bi].wide || blocks[bi + 1].wide || (*second)[bi]) continue;
        uint64_t T = blocks[bi].qmask | blocks[bi + 1].qmask | 1ull;
        if (__builtin_popcountll(T) > 12) continue;
        for (int extra = 0; extra < n && __builtin_popcountll(T) < 12; ++extra) T |= 1ull << extra;
        (*tileset)[bi] = T;
        (*second)[bi + 1] = 1;
    }
}

// the planner depth the fused plan runs with, and the cheaper one the learned
// plan uses to predict block counts for its features
constexpr int kRunDepth = 3;
constexpr size_t kFirstGroup = 2;   // blocks of the first group (planned at depth <= 2)
constexpr size_t kGroupBlocks = 8;  // blocks of every later group
constexpr int kFeatureDepth = 1;

// CTAs of one kernel that fit on an SM at once: registers (allocated per warp
// in units of 256), shared memory (static + dynamic + the per-CTA reservation)
// and threads.
int resident_ctas(int dev, const void *fn, int threads, size_t dyn_smem)
{
    cudaFuncAttributes fa{};
    int regs_sm = 0, smem_sm = 0, smem_rsv = 0, thr_sm = 0;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return 0;
    const int warps = (threads + 31) / 32;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_warp > 0 ? (regs_sm / regs_warp) / warps : 0;
    const size_t smem_cta = fa.sharedSizeBytes + dyn_smem + (size_t)smem_rsv;
    const int by_smem = (int)((size_t)smem_sm / smem_cta);
    const int by_thr = thr_sm / (warps * 32);
    return std::min(by_regs, std::min(by_smem, by_thr));
}

// The spectral norm of one lowered gate as an operator on the register (a
// controlled gate is the identity where a control is 0): an upper bound on
// how much it can raise the state's norm.
static double sgate_norm_bound(const SGate &g)
{
    const double *u = g.m;
    const double f2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2] + u[3] * u[3] + u[4] * u[4] + u[5] * u[5] +
                      u[6] * u[6] + u[7] * u[7];
    // det = A D - B C
    const double dr = (u[0] * u[6] - u[1] * u[7]) - (u[2] * u[4] - u[3] * u[5]);
    const double di = (u[0] * u[7] + u[1] * u[6]) - (u[2] * u[5] + u[3] * u[4]);
    // sigma_max^2 = (|G|_F^2 + sqrt(|G|_F^4 - 4 |det|^2)) / 2
    const double disc = std::max(f2 * f2 - 4.0 * (dr * dr + di * di), 0.0);
    const double sig = std::sqrt(0.5 * (f2 + std::sqrt(disc)));
    return g.ctrl ? std::max(sig, 1.0) : sig;
}

// k = 6: the exponent we of the power-of-two scale of a block's W, and the
// block's norm bound (every entry of U_blk = G_m ... G_1, and so of its real
// form W, is at most the spectral norm of U_blk, which is at most the product
// of its gates' spectral norms).  we = 14 - ceil(log2 bound) keeps |2^we W| <=
// 2^14 (1 + 1e-6), far below the FP16 maximum; a unitary block gets 14.  we
// lies in [kF16WExpMin, kF16WExpMax]; returns false when the bound is too
// large (above 2^114) or not finite.
// a bound on the spectral norm of a 4 x 4 matrix S (32 doubles, row-major
// (re, im)): sqrt(||S||_1 ||S||_inf) (Hoelder), exactly 1 for the
// depolarizing, phase-damping and flip channels
static double super_norm_bound(const double *S)
{
    double c1 = 0.0, ci = 0.0;
    for (int i = 0; i < 4; ++i) {
        double row = 0.0, col = 0.0;
        for (int j = 0; j < 4; ++j) {
            row += std::hypot(S[2 * (4 * i + j)], S[2 * (4 * i + j) + 1]);
            col += std::hypot(S[2 * (4 * j + i)], S[2 * (4 * j + i) + 1]);
        }
        ci = std::max(ci, row);
        c1 = std::max(c1, col);
    }
    return std::sqrt(c1 * ci);
}

static double member_norm_bound(const SGate &g, const double *sup)
{
    return g.op == OP_SUPER ? super_norm_bound(sup + 32 * (size_t)g.orig) : sgate_norm_bound(g);
}

static bool block_wexp(const std::vector<SGate> &g, const std::vector<int> &members, int *we, double *bound_out,
                       const double *sup)
{
    double bound = 1.0;
    for (int m : members) bound *= member_norm_bound(g[m], sup);
    *bound_out = bound;
    if (!std::isfinite(bound)) return false;
    int eb = 0;
    if (bound > 1.0 + 1e-6)
        eb = (int)std::ceil(std::log2(bound / (1.0 + 1e-6)));
    else if (bound < 1.0)
        eb = bound > 0.0 ? std::max((int)std::ceil(std::log2(bound)), kF16WExp - kF16WExpMax)
                         : kF16WExp - kF16WExpMax;
    const int w = kF16WExp - eb;
    if (w < kF16WExpMin) return false;
    *we = std::min(w, kF16WExpMax);
    return true;
}

// Plan and run the fused blocks in groups: each group of blocks is planned,
// its gates uploaded, its W matrices built (one k_fuse_build launch) and its
// applies launched; the host then plans the next group while the GPU works
// through this one, so only the first (small) group's planning is exposed.
// Host and device copies of the gate lists keep one region per group (no
// reuse within a call); the W matrices use two device slots, reused in
// stream order.
template <int KQ>
int run_fused(qsim_state *s, const std::vector<SGate> &g, int depth, bool allow_multi, const double *sup = nullptr)
{
    constexpr int K = 2 << KQ;
    constexpr size_t kGroup = kGroupBlocks;
    constexpr size_t kFirst = kFirstGroup;
    const int n = s->n;
    size_t ng = g.size();
    for (const SGate &x : g)
        if (x.op == OP_SUPER) ng += 3;             // a 4 x 4 takes four block-gate records
    // complex128 (k = 4 only): the integer digit-plane kernels of fused64.cu
    const bool c128 = s->dtype == SIM_C128;
    const size_t blk_bytes = c128 ? fused_c128_slot_bytes() : 2 * (size_t)K * K * sizeof(float);
    // per call: gate lists (<= ng FGates, <= 2 ng + 1 offsets), W slots (2 x kGroup blocks)
    const size_t bytes_g = ng * sizeof(FGate), bytes_o = (2 * ng + 2) * sizeof(int), bytes_e = (ng + 1) * sizeof(int);
    const size_t bytes_slot = kGroup * blk_bytes;
    const size_t o_g = 0, o_o = (bytes_g + 255) & ~(size_t)255, o_e = (o_o + bytes_o + 255) & ~(size_t)255,
                 o_w = (o_e + bytes_e + 255) & ~(size_t)255;
    const size_t total = o_w + 2 * bytes_slot;
    if (int rc = ensure_host_pinned(&s->host_ops, &s->host_ops_bytes, o_w)) return rc;
    char *scratch = nullptr;
    QSIM_CUDA(cudaMallocAsync((void **)&scratch, total, s->stream));
    FGate *hg = (FGate *)((char *)s->host_ops + o_g);
    int *ho = (int *)((char *)s->host_ops + o_o);
    int *he = (int *)((char *)s->host_ops + o_e);    // per block: W exponent (k = 6)
    size_t be_used = 0;
    double growth = 1.0;                             // k = 6: bound on norm^2 growth so far in this call
    std::vector<double> bnd;                         // k = 6: per block of the group, its norm bound
    int rc = SIM_OK;
    do {
        if (cudaMemsetAsync(s->dev_status, 0, sizeof(int), s->stream) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "status reset");
            break;
        }
        // k = 6: the state's norm^2 on the device (one pass over the state,
        // overlapping the host's planning of the first group); the blocks
        // derive their FP16 scale from it
        if (KQ == 6 && (rc = reduce_norm_device(s)) != SIM_OK) break;
        // shared-memory limits and carveouts of the kernels this plan launches
        auto attrs = [](const void *fn, size_t dyn) {
            return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) == cudaSuccess &&
                   cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared) == cudaSuccess;
        };
        const size_t smb = (size_t)(1 << KQ) * ((1 << KQ) / kBuildSplit<KQ>) * sizeof(double2);
        if (!attrs((const void *)k_fuse_build<KQ>, smb)) {
            rc = cuda_fail(cudaGetLastError(), "fused kernel attributes");
            break;
        }
        const uint64_t rows = 1ull << (n - KQ);
        // k <= 5: the persistent streamed kernel, as many CTAs as fit at once
        // (k = 6 does not fit W, a stage ring and A in shared memory)
        int pipe_grid = 0;
        size_t smp = 0;
        if (c128) {
            if ((rc = fused_c128_prepare(s, &pipe_grid)) != SIM_OK) break;
        } else if constexpr (KQ <= 5) {
            smp = stream_smem_bytes<KQ>();
            if (!attrs((const void *)k_fused_stream<KQ>, smp)) {
                rc = cuda_fail(cudaGetLastError(), "streamed kernel attributes");
                break;
            }
            // CTAs per SM from the kernel's own register and shared-memory
            // footprint; the CTAs never wait on one another, so this only
            // sets the grid
            int per_sm = resident_ctas(s->device, (const void *)k_fused_stream<KQ>, kStreamThreads, smp);
            if (per_sm < 1) {
                rc = fail(SIM_ECUDA, "fused apply: streamed kernel does not fit on an SM");
                break;
            }
            const int cols = 4 * (2 << KQ);                              // TMEM columns per CTA
            per_sm = std::min(per_sm, 512 / cols);
            const uint64_t tiles = (rows + kRows - 1) / kRows;
            pipe_grid = (int)std::min<uint64_t>(tiles, (uint64_t)s->num_sms * per_sm);
        } else {
            // k = 6: one CTA per SM (all of tensor memory, 192 KB of shared memory)
            smp = tmem6_smem_bytes();
            if (!attrs((const void *)k_fused_tmem6, smp)) {
                rc = cuda_fail(cudaGetLastError(), "k = 6 kernel attributes");
                break;
            }
            if (resident_ctas(s->device, (const void *)k_fused_tmem6, kT6Threads, smp) < 1) {
                rc = fail(SIM_ECUDA, "fused apply: the k = 6 kernel does not fit on an SM");
                break;
            }
            const uint64_t tiles = (rows + kRows - 1) / kRows;
            pipe_grid = (int)std::min<uint64_t>(tiles, (uint64_t)s->num_sms);
        }
        // the first group is planned at depth <= 2 (its planning time is exposed)
        int multi_grid = 0;
        size_t smm = 0;
        const bool multi = KQ == 5 && n >= 12 && allow_multi && !c128;
        if (multi) {
            smm = multi_smem_bytes(kMaxPass);
            if (!attrs((const void *)k_fused_multi, smm)) {
                rc = cuda_fail(cudaGetLastError(), "multi-block kernel attributes");
                break;
            }
            const uint64_t tiles = (rows + kRows - 1) / kRows;
            multi_grid = (int)std::min<uint64_t>(tiles, (uint64_t)s->num_sms);
        }
        BlockPlanner planner(g, KQ, n, std::min(depth, 2));
        size_t fg_used = 0, go_used = 0;
        int slot = 0;
        for (size_t grp = 0; rc == SIM_OK; ++grp, slot ^= 1) {
            // plan the next group
            std::vector<Block> blocks;
            Block b;
            const size_t want = grp == 0 ? kFirst : kGroup;
            while (blocks.size() < want && planner.next(&b)) blocks.push_back(b);
            if (blocks.empty()) break;
            if (grp == 0) planner.set_depth(depth);
            // k = 5: consecutive pairs of blocks whose qubits, with qubit 0,
            // fit one 12-qubit tile run as one multi-block pass
            std::vector<uint64_t> tileset;   // T of the pass a block opens, 0 = single
            std::vector<char> second;        // block runs inside the previous block's pass
            pair_blocks(blocks, n, KQ == 5 && multi, &tileset, &second);
            // pad every block to KQ qubits (identity on the added ones): a block
            // of a pass pads with qubits of the pass's tile, others with the
            // lowest qubits; gates in block-local qubits
            const size_t fg0 = fg_used, go0 = go_used, be0 = be_used;
            std::vector<std::vector<int>> pos(blocks.size());
            bnd.assign(blocks.size(), 1.0);
            ho[go_used++] = 0;
            for (size_t bi = 0; bi < blocks.size() && rc == SIM_OK; ++bi) {
                int we = kF16WExp;
                if (KQ == 6 && !block_wexp(g, blocks[bi].members, &we, &bnd[bi], sup))
                    rc = fail(SIM_EUNSUPPORTED, "fused apply, k = 6: the product of a block's gate norms is above "
                                                "2^114 or not finite (beyond the range of its FP16 scale)");
                he[be_used++] = we;
                if (!blocks[bi].wide) {
                    uint64_t q = blocks[bi].qmask;
                    const uint64_t T = tileset[bi] ? tileset[bi] : (second[bi] ? tileset[bi - 1] : ~0ull);
                    for (int extra = 0; extra < n && __builtin_popcountll(q) < KQ; ++extra)
                        if ((T >> extra) & 1) q |= 1ull << extra;
                    for (int i = 0; i < n; ++i)
                        if ((q >> i) & 1) pos[bi].push_back(i);
                    auto loc = [&](int qubit) {
                        for (int i = 0; i < KQ; ++i)
                            if (pos[bi][i] == qubit) return i;
                        return -1;
                    };
                    for (int m : blocks[bi].members) {
                        if (g[m].op == OP_SUPER) {
                            const double *S = sup + 32 * (size_t)g[m].orig;
                            for (int l = 0; l < 4; ++l) {
                                FGate f;
                                f.target = l == 0 ? kSuperHead : kSuperRow;
                                f.ctrl = l == 0 ? ((uint32_t)loc(g[m].target) | ((uint32_t)loc(g[m].target2) << 8)) : 0u;
                                memcpy(f.m, S + 8 * l, sizeof f.m);
                                hg[fg_used++] = f;
                            }
                            continue;
                        }
                        FGate f;
                        f.target = loc(g[m].target);
                        f.ctrl = 0;
                        for (int c = 0; c < n; ++c)
                            if ((g[m].ctrl >> c) & 1) f.ctrl |= 1u << loc(c);
                        memcpy(f.m, g[m].m, sizeof f.m);
                        hg[fg_used++] = f;
                    }
                }
                ho[go_used++] = (int)(fg_used - fg0);
            }
            if (rc != SIM_OK) break;
            const size_t nb = blocks.size();
            FGate *dg = (FGate *)(scratch + o_g) + fg0;
            int *dgo = (int *)(scratch + o_o) + go0;
            int *dge = (int *)(scratch + o_e) + be0;
            float *dw = (float *)(scratch + o_w + (size_t)slot * bytes_slot);
            char *dwb = (char *)dw;
            if ((fg_used > fg0 && cudaMemcpyAsync(dg, hg + fg0, (fg_used - fg0) * sizeof(FGate), cudaMemcpyHostToDevice,
                                                  s->stream) != cudaSuccess) ||
                cudaMemcpyAsync(dgo, ho + go0, (nb + 1) * sizeof(int), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
                (KQ == 6 &&
                 cudaMemcpyAsync(dge, he + be0, nb * sizeof(int), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)) {
                rc = cuda_fail(cudaGetLastError(), "fused upload");
                break;
            }
            if (c128) {
                if ((rc = launch_fuse_build_c128(s, dg, dgo, (int)nb, dwb))) break;
            } else {
                launch_begin(s, KC_FUSE_BUILD, (double)nb * 2 * K * K * sizeof(float));
                k_fuse_build<KQ><<<(unsigned)(nb * kBuildSplit<KQ>), 256, smb, s->stream>>>(dg, dgo, dge, dw);
                if ((rc = launch_end(s, "fused build"))) break;
            }
            for (size_t bi = 0; bi < nb && rc == SIM_OK; ++bi) {
                if (blocks[bi].wide) {
                    rc = launch_sgate(s, g[blocks[bi].members[0]]);
                    const double b = sgate_norm_bound(g[blocks[bi].members[0]]);
                    growth *= b * b;
                    continue;
                }
                if constexpr (KQ == 5) {
                    if (tileset[bi]) {
                        // blocks bi, bi + 1 in one pass
                        PassArgs pa{};
                        pa.m = 2;
                        for (int i = 0, t = 0; i < n; ++i)
                            if ((tileset[bi] >> i) & 1) pa.tpos[t++] = i;
                        for (int j = 0; j < 2; ++j)
                            for (int i = 0; i < KQ; ++i) pa.pos[j][i] = pos[bi + j][i];
                        launch_begin(s, KC_FUSED_MULTI, 2.0 * (double)s->bytes, 2 * 3.0 * 2.0 * (double)rows * K * K);
                        k_fused_multi<<<(unsigned)multi_grid, kMultiThreads, smm, s->stream>>>(
                            (float *)s->amps, dw + bi * 2 * (size_t)K * K, pa, (rows + kRows - 1) / kRows,
                            s->dev_status);
                        rc = launch_end(s, "fused multi-block pass");
                        ++bi;
                        continue;
                    }
                }
                if (c128) {
                    rc = launch_fused_c128(s, dwb + bi * blk_bytes, pos[bi].data(), pipe_grid);
                    continue;
                }
                ApplyArgs a{};
                a.nq = KQ;
                for (int i = 0; i < KQ; ++i) a.pos[i] = pos[bi][i];
                a.rows = rows;
                a.wexp = he[be0 + bi];
                a.nrm2 = s->red_out;
                a.growth = growth;
                growth *= bnd[bi] * bnd[bi];
                // tensor-core flops: three real GEMMs [rows x K] x [K x K] (3xTF32; k = 6: FP16 split)
                launch_begin(s, KQ <= 5 ? KC_FUSED : KC_FUSED_F16, 2.0 * (double)s->bytes,
                             3.0 * 2.0 * (double)rows * K * K);
                const float *bm = dw + bi * 2 * (size_t)K * K;
                if constexpr (KQ <= 5) {
                    k_fused_stream<KQ><<<(unsigned)pipe_grid, kStreamThreads, smp, s->stream>>>(
                        (float *)s->amps, bm, a, (rows + kRows - 1) / kRows, s->dev_status);
                } else {
                    k_fused_tmem6<<<(unsigned)pipe_grid, kT6Threads, smp, s->stream>>>(
                        (float *)s->amps, reinterpret_cast<const __half *>(bm), a, (rows + kRows - 1) / kRows,
                        s->dev_status);
                }
                rc = launch_end(s, "fused apply");
            }
        }
    } while (0);
    cudaFreeAsync(scratch, s->stream);
    int hstatus = 0;
    QSIM_CUDA(cudaMemcpyAsync(&hstatus, s->dev_status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    QSIM_CUDA(cudaStreamSynchronize(s->stream));
    if (rc == SIM_OK && hstatus != 0)
        rc = fail(SIM_ETIMEOUT, "fused apply: a tensor-core wait gave up");
    return rc;
}

}  // namespace

int describe_fused(int n, const sim_gate *gates, size_t n_gates, int k, int64_t *blocks_out, int depth, bool multi,
                   int64_t *passes_out)
{
    std::vector<SGate> g;
    lower_gates(gates, n_gates, &g);
    // the same schedule as the run: the first group's blocks at depth <= 2
    const int d = depth > 0 ? depth : kRunDepth;
    BlockPlanner planner(g, k, n, std::min(d, 2));
    int64_t nb = 0, np = 0;
    for (size_t grp = 0;; ++grp) {
        std::vector<Block> blocks;
        Block b;
        const size_t want = grp == 0 ? kFirstGroup : kGroupBlocks;
        while (blocks.size() < want && planner.next(&b)) blocks.push_back(b);
        if (blocks.empty()) break;
        if (grp == 0) planner.set_depth(d);
        std::vector<uint64_t> tileset;
        std::vector<char> second;
        pair_blocks(blocks, n, k == 5 && multi, &tileset, &second);
        nb += (int64_t)blocks.size();
        for (size_t i = 0; i < blocks.size(); ++i) np += second[i] ? 0 : 1;
    }
    if (blocks_out) *blocks_out = nb;
    if (passes_out) *passes_out = np;
    return SIM_OK;
}

int fused_feature_depth() { return kFeatureDepth; }

int apply_sgates_fused(qsim_state *s, const std::vector<SGate> &g, const double *sup, int k)
{
    if (k < 3 || k > 6) return fail(SIM_EINVAL, "fused plan: fuse_k must be in 3..6");
    if (s->dtype == SIM_C128 && k != 4)
        return fail(SIM_EUNSUPPORTED, "fused plan: complex128 states run 4-qubit blocks (fuse_k 4 or 0)");
    if (s->n < k + 7) return fail(SIM_EINVAL, "fused plan: needs n >= fuse_k + 7 (one CTA covers 128 rows)");
    if (g.empty()) return SIM_OK;
    switch (k) {
    case 3: return run_fused<3>(s, g, kRunDepth, false, sup);
    case 4: return run_fused<4>(s, g, kRunDepth, false, sup);
    case 5: return run_fused<5>(s, g, kRunDepth, false, sup);
    default: return run_fused<6>(s, g, kRunDepth, false, sup);
    }
}

int apply_circuit_fused(qsim_state *s, const sim_gate *gates, size_t n_gates, const sim_plan_opts &o)
{
    const bool c128 = s->dtype == SIM_C128;
    int k = o.fuse_k ? o.fuse_k : (c128 ? 4 : 5);
    if (k < 3 || k > 6) return fail(SIM_EINVAL, "fused plan: fuse_k must be in 3..6");
    if (c128 && k != 4) return fail(SIM_EUNSUPPORTED, "fused plan: complex128 states run 4-qubit blocks (fuse_k 4 or 0)");
    if (s->n < k + 7) return fail(SIM_EINVAL, "fused plan: needs n >= fuse_k + 7 (one CTA covers 128 rows)");
    std::vector<SGate> g;
    lower_gates(gates, n_gates, &g);
    if (g.empty()) return SIM_OK;
    const bool multi = (o.flags & SIM_FLAG_MULTI_BLOCK_PASSES) != 0;
    switch (k) {
    case 3: return run_fused<3>(s, g, kRunDepth, multi);
    case 4: return run_fused<4>(s, g, kRunDepth, multi);
    case 5: return run_fused<5>(s, g, kRunDepth, multi);
    default: return run_fused<6>(s, g, kRunDepth, multi);
    }
}

}  // namespace qsim
