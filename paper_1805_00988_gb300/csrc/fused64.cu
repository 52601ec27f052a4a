// fused64.cu -- complex128 fused blocks on the tensor cores.
//
// A fused block is the product of its gates restricted to k qubits (§1.3.2:
// U_t = I (x) ... (x) U (x) ... (x) I restricted to the block's qubits), applied
// to the state as the real GEMM D = X W described in fused.cu.  For complex128
// states the GEMM must be exact to FP64 level, and this GPU's FP64 pipe is
// narrow, so the products run on the FP16 tensor cores as exact integer
// arithmetic, after the error-free splitting of Ozaki, Ogita, Oishi and Rump
// (2012), in the fixed-point form used on tensor cores by Mukunoki, Ozaki,
// Ogita and Imamura (2020):
//   - each row r of X (the 2^k amplitudes sharing all index bits outside the
//     block, as 2^(k+1) reals) is written in fixed point relative to its
//     largest component: |x| < 2^E_r, t = trunc(x 2^(47 - E_r)), |t| < 2^47,
//     and t is cut into kPlanes = 6 balanced base-256 digits, t = sum_i d_i
//     256^(5 - i) with |d_i| <= 128: the bytes of |t| + 128 (1 + 256 + ... +
//     256^5), each less 128 (digit 0 from bits 40 and up), times x's sign;
//   - each column n of W likewise relative to its largest entry (2^F_n);
//   - a digit is an integer of magnitude at most 128, exact in FP16, and a
//     product of two is at most 2^14; a K = 32 sum of them is at most 2^19,
//     and the products of digit i of X with digit j of W are summed per
//     level l = i + j (at most 6 products per level, below 2^22), so every
//     FP32 accumulator holds an exact integer (the tensor core adds integers
//     below 2^24 without rounding);
//   - levels l = 0..5 are kept (pairs with i + j >= 6 are dropped, a relative
//     error of about 2^-42 of the row and column maxima in the worst case),
//     and the consumer forms T = sum_l D_l 256^(5 - l) exactly in 64-bit
//     integers, converts it to FP64 (rounded to nearest) and scales it by
//     2^(E_r + F_n - 54).
// One MMA per digit plane i of X and K-step: A = plane i (128 rows x 16), B =
// W's planes 0 .. 5 - i side by side (N = (6 - i) x 32), D = accumulator
// columns of levels i .. 5, so levels accumulate in place: 12 MMAs per tile.
//
// k = 4 (K = N = 32 per level): two accumulators of 6 x 32 columns fit in
// tensor memory, the six digit planes of A in shared memory.
//   warp 17: loads tile i (128 rows x 16 amplitudes, runs of >= 2 KB) into
//       stage i mod 3 with bulk copies (three tiles in flight);
//   warps 0-7: threads 2 r and 2 r + 1 turn row r into its exponent and digit
//       planes (A buffer i mod 2, K-major FP16), half of its columns each,
//       once the MMAs of tile i - 2 are done;
//   warp 16 (one thread): the 12 MMAs of tile i once A is written and
//       accumulator i mod 2 has been drained (tile i - 2);
//   warps 8-15: a thread per row and half of the columns reads the row's
//       levels (4-column chunks, the next chunk's loads in flight while the
//       current one is converted), forms the FP64 results and stores them.
// The integer work (digit split, level recombination) sets this kernel's
// pace, so it is spread over 512 threads (at most 112 registers each) rather
// than 256: more warps to issue from while others wait on shared memory or
// tensor memory.
// Row exponents pass from converter to consumer through four shared-memory
// slots with their own full / empty barriers.  Every wait is bounded; on a
// timeout the kernel records SIM_ETIMEOUT, lets work in flight land (bounded
// again), frees its tensor memory and returns.
#include <cstring>

#include <cuda_fp16.h>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace qsim {

namespace {

constexpr int kQ64 = 4;                       // qubits per block
constexpr int kD64 = 1 << kQ64;               // amplitudes per row
constexpr int kK64 = 2 * kD64;                // reals per row: MMA K, and N per level
constexpr int kPlanes = 6;                    // balanced base-256 digits per operand
constexpr int kRows64 = 128;                  // MMA M, rows per tile
constexpr int kTB64 = kQ64 + 7;               // tile bits
constexpr int kTAmp64 = 1 << kTB64;           // amplitudes per tile
constexpr int kT64Threads = 576;            // 8 converter + 8 consumer warps, issuer, loader
constexpr int kHalf64 = 2 * kRows64;         // converter (and consumer) threads: two per row
constexpr uint32_t kPlaneB = (uint32_t)kK64 * kK64 * 2;            // one W plane: 32 x 32 halves
constexpr uint32_t kAPlaneB = (uint32_t)kRows64 * kK64 * 2;         // one A plane: 128 x 32 halves
constexpr uint32_t kSlot64 = kPlanes * kPlaneB + kK64 * sizeof(int); // per block: W planes + column exponents
constexpr int kSe64 = 4;                      // row-exponent slots
constexpr int kStage64 = 3;                   // tiles in flight from HBM

struct FGate64 {                              // a gate in block-local qubits (the host's block-gate layout)
    int32_t target;
    uint32_t ctrl;
    double m[8];
};

struct Apply64 {
    int pos[kQ64];                            // global qubits of the block, ascending
};

__device__ __forceinline__ void mma_f16_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accum)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void tmem_ld4_nowait(uint32_t taddr, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
}
// tcgen05.wait::ld that also names the 24 registers of one chunk as read and
// written, so no use of them can be scheduled above the wait
__device__ __forceinline__ void tmem_wait_ld_regs(uint32_t (&r)[6][4])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0][0]), "+r"(r[0][1]), "+r"(r[0][2]), "+r"(r[0][3]), "+r"(r[1][0]), "+r"(r[1][1]),
                   "+r"(r[1][2]), "+r"(r[1][3]), "+r"(r[2][0]), "+r"(r[2][1]), "+r"(r[2][2]), "+r"(r[2][3]),
                   "+r"(r[3][0]), "+r"(r[3][1]), "+r"(r[3][2]), "+r"(r[3][3]), "+r"(r[4][0]), "+r"(r[4][1]),
                   "+r"(r[4][2]), "+r"(r[4][3]), "+r"(r[5][0]), "+r"(r[5][1]), "+r"(r[5][2]), "+r"(r[5][3])
                 :
                 : "memory");
}

// biased FP64 exponent of a component (0 for zero and subnormals, which are
// taken as zero)
__device__ __forceinline__ uint32_t bexp(double x) { return (uint32_t)(__double_as_longlong(x) >> 52) & 0x7FFu; }

// 128 (1 + 256 + ... + 256^5): added to t, it leaves digit i + 128 in byte
// 5 - i (digit 0: bits 40 and up, 0..256)
constexpr uint64_t kDigitOff = 0x808080808080ull;

// t + kDigitOff with t = trunc(|x| 2^(47 - E)), E = emax - 1022 the exponent
// bound of x's row or column (|x| < 2^E, emax the largest biased exponent),
// so 0 <= t < 2^47; x given as its two 32-bit halves.  Zero and subnormal x
// give t = 0 (their shift is 64; PTX clamps 64-bit shifts at 64).  The
// balanced digits of t, each times the sign of x, are those of x 2^(47 - E).
__device__ __forceinline__ uint64_t fixed47m(uint32_t hi, uint32_t lo, uint32_t emax)
{
    const uint32_t e = (hi >> 20) & 0x7FFu;
    const uint32_t sh = e ? emax - e + 6u : 64u;        // >= 6
    const uint64_t m = ((uint64_t)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
    uint64_t t;
    asm("shr.b64 %0, %1, %2;" : "=l"(t) : "l"(m), "r"(sh));
    return t + kDigitOff;
}

// ------------------------------------------------------------------ builder
// U = G_m ... G_1 in FP64 (columns evolved from the identity), then its real
// form W (fused.cu's convention), each column n in fixed point relative to
// its largest entry, cut into kPlanes balanced digit planes (FP16, exact) in the 16-bit K-major
// B-operand layout ([plane][n][kk], plane j as rows 32 j .. 32 j + 31), and the
// columns' biased exponents after the planes.  One CTA per block.
__global__ void __launch_bounds__(256) k_fuse_build64(const FGate64 *__restrict__ gates, const int *__restrict__ goff,
                                                      unsigned char *__restrict__ bout)
{
    constexpr int D = kD64, K = kK64;
    __shared__ double2 U[D][D];               // U[i][c]: row i, column c
    __shared__ uint32_t cmax[K];
    const int blk = blockIdx.x, tid = threadIdx.x;
    for (int e = tid; e < D * D; e += 256) U[e / D][e % D] = make_double2((e / D) == (e % D) ? 1.0 : 0.0, 0.0);
    if (tid < K) cmax[tid] = 0;
    __syncthreads();
    for (int g = goff[blk]; g < goff[blk + 1]; ++g) {
        const int t = gates[g].target;
        const uint32_t cm = gates[g].ctrl;
        if (t == -1) {
            // a 4 x 4 matrix on local qubits la < lb in four records (rows of S,
            // l = 2 (bit lb) + (bit la); the block-gate layout of fused.cu)
            const int la = (int)(cm & 0xFFu), lb = (int)((cm >> 8) & 0xFFu);
            for (int e = tid; e < D * (D / 4); e += 256) {
                const int c = e / (D / 4);
                int i0 = e % (D / 4);
                i0 = ((i0 >> la) << (la + 1)) | (i0 & ((1 << la) - 1));
                i0 = ((i0 >> lb) << (lb + 1)) | (i0 & ((1 << lb) - 1));
                const int idx[4] = {i0, i0 | (1 << la), i0 | (1 << lb), i0 | (1 << la) | (1 << lb)};
                double2 x[4];
#pragma unroll
                for (int l = 0; l < 4; ++l) x[l] = U[idx[l]][c];
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const double *r = gates[g + l].m;
                    double yr = 0.0, yi = 0.0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        yr += r[2 * k] * x[k].x - r[2 * k + 1] * x[k].y;
                        yi += r[2 * k] * x[k].y + r[2 * k + 1] * x[k].x;
                    }
                    U[idx[l]][c] = make_double2(yr, yi);
                }
            }
            __syncthreads();
            g += 3;
            continue;
        }
        const double ar = gates[g].m[0], ai = gates[g].m[1], br = gates[g].m[2], bi = gates[g].m[3];
        const double cr = gates[g].m[4], ci = gates[g].m[5], dr = gates[g].m[6], di = gates[g].m[7];
        for (int e = tid; e < D * (D / 2); e += 256) {
            const int c = e / (D / 2), p = e % (D / 2);
            const int i0 = ((p >> t) << (t + 1)) | (p & ((1 << t) - 1));
            if (((uint32_t)i0 & cm) != cm) continue;
            const int i1 = i0 | (1 << t);
            const double2 a = U[i0][c], b = U[i1][c];
            U[i0][c] = make_double2(ar * a.x - ai * a.y + br * b.x - bi * b.y, ar * a.y + ai * a.x + br * b.y + bi * b.x);
            U[i1][c] = make_double2(cr * a.x - ci * a.y + dr * b.x - di * b.y, cr * a.y + ci * a.x + dr * b.y + di * b.x);
        }
        __syncthreads();
    }
    // W[kk][n]: input kk = 2 j + a, output n = 2 i + b
    auto wval = [&](int n, int kk) {
        const int i = n >> 1, b = n & 1, j = kk >> 1, a = kk & 1;
        const double2 u = U[i][j];
        return (a == b) ? u.x : (a == 1 ? -u.y : u.y);
    };
    for (int e = tid; e < K * K; e += 256) atomicMax(&cmax[e / K], bexp(wval(e / K, e % K)));
    __syncthreads();
    unsigned char *out = bout + (size_t)blk * kSlot64;
    for (int e = tid; e < K * K; e += 256) {
        const int n = e / K, kk = e % K;
        const double w = wval(n, kk);
        const uint64_t t = fixed47m((uint32_t)__double2hiint(w), (uint32_t)__double2loint(w), cmax[n]);
        for (int p = 0; p < kPlanes; ++p) {
            // digit p: byte 5 - p of t + kDigitOff (digit 0: bits 40 and up) less 128, with w's sign
            const int dm = (int)(p == 0 ? (t >> 40) : ((t >> (40 - 8 * p)) & 255u)) - 128;
            const int d = (w < 0.0) ? -dm : dm;
            *reinterpret_cast<__half *>(out + kmajor16_off((uint32_t)(p * K + n), (uint32_t)kk, K)) = __int2half_rn(d);
        }
    }
    if (tid < K) reinterpret_cast<int *>(out + kPlanes * kPlaneB)[tid] = (int)cmax[tid];
}

// ------------------------------------------------------------------ apply
__global__ void __launch_bounds__(kT64Threads, 1)
    k_fused_c128(double *__restrict__ st, const unsigned char *__restrict__ bblk, Apply64 a, uint64_t ntiles,
                 int *__restrict__ status)
{
    constexpr int D = kD64, K = kK64, TB = kTB64, TAMP = kTAmp64;
    constexpr uint32_t TBYTES = (uint32_t)TAMP * 16u;
    constexpr uint32_t NCOLS = 512, ACC = 256;          // accumulator b at column 256 b (6 x 32 used)
    constexpr uint32_t SBO = (K / 8) * 128;             // 8-row group stride of a 16-bit K-major operand

    extern __shared__ __align__(1024) unsigned char smem[];
    double2 *stage = reinterpret_cast<double2 *>(smem);                          // kStage64 x TAMP amplitudes
    unsigned char *abuf = smem + kStage64 * (size_t)TBYTES;                              // 2 x 6 planes x 128 x 32 halves
    unsigned char *wsm = abuf + 2 * (size_t)kPlanes * kAPlaneB;                   // 6 planes x 32 x 32 halves
    __shared__ uint64_t bar_full[kStage64], bar_empty[kStage64], bar_a[2], bar_d[2], bar_e[2], bar_sf[kSe64], bar_se[kSe64];
    __shared__ uint32_t rowexp[kSe64][kRows64];
    __shared__ int colexp[K];
    __shared__ uint32_t tslot;
    __shared__ int tpos[TB];
    __shared__ uint64_t pmask;
    __shared__ int lrun;
    __shared__ uint32_t uc[D];
    __shared__ uint64_t gc[D];
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        failed = *reinterpret_cast<volatile int *>(status);
        uint64_t pm = 0;
        for (int i = 0; i < kQ64; ++i) pm |= 1ull << a.pos[i];
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
        for (int b = 0; b < kStage64; ++b) {
            mbar_init(&bar_full[b], 1);
            mbar_init(&bar_empty[b], kHalf64);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar_a[b], kHalf64);
            mbar_init(&bar_d[b], 1);
            mbar_init(&bar_e[b], kHalf64);
        }
        for (int q = 0; q < kSe64; ++q) {
            mbar_init(&bar_sf[q], kHalf64);
            mbar_init(&bar_se[q], kHalf64);
        }
    }
    for (int c = tid; c < D; c += kT64Threads) {
        uint32_t u = 0;
        uint64_t g = 0;
        for (int i = 0; i < kQ64; ++i)
            if ((c >> i) & 1) {
                g |= 1ull << a.pos[i];
                for (int j = 0; j < TB; ++j)
                    if (tpos[j] == a.pos[i]) u |= 1u << j;
            }
        uc[c] = u;
        gc[c] = g;
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(bblk);
        uint4 *dst = reinterpret_cast<uint4 *>(wsm);
        for (int e = tid; e < (int)(kPlanes * kPlaneB / 16); e += kT64Threads) dst[e] = __ldg(src + e);
        if (tid < K) colexp[tid] = reinterpret_cast<const int *>(bblk + kPlanes * kPlaneB)[tid];
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

    if (warp == 17) {
        // loader: lane j copies run j of every tile (T holds qubits 0..6, so
        // runs are >= 128 amplitudes and a tile has at most 16 of them)
        const int L = lrun;
        const int nrun = 1 << (TB - L);
        const uint32_t rbytes = 16u << L;
        int issued = 0;
        for (int i = 0; i < iters && !warp_flag(vfailed); ++i) {
            const int s = i % kStage64;
            if (i >= kStage64 && !mbar_wait_warp(&bar_empty[s], (uint32_t)((i / kStage64 - 1) & 1))) {
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
        if (lane == 0)
            for (int i = (issued > kStage64 ? issued - kStage64 : 0); i < issued; ++i)
                mbar_wait_bounded(&bar_full[i % kStage64], (uint32_t)((i / kStage64) & 1));
    } else if (warp < 8) {
        // converters: threads 2 r and 2 r + 1 share row r, each taking half of
        // its complex columns (one shuffle gives both the row's exponent)
        const int r = tid >> 1, h = tid & 1;
        uint32_t ur;
        uint64_t gr;
        row_offsets(r, ur, gr);
        const uint32_t arow = (((uint32_t)r >> 3) * (K >> 3) << 7) + (((uint32_t)r & 7) << 4);
        constexpr int DH = D / 2;
        for (int i = 0; i < iters && !warp_flag(vfailed); ++i) {
            const int s = i % kStage64, b = i & 1;
            if (!mbar_wait_warp(&bar_full[s], (uint32_t)((i / kStage64) & 1))) {
                *vfailed = 1;
                break;
            }
            const double2 *sg = stage + (size_t)s * TAMP;
            double2 v[DH];
#pragma unroll
            for (int c = 0; c < DH; ++c) v[c] = sg[ur | uc[DH * h + c]];
            mbar_arrive(&bar_empty[s]);
            uint32_t emax = 0;
#pragma unroll
            for (int c = 0; c < DH; ++c) emax = max(emax, max(bexp(v[c].x), bexp(v[c].y)));
            emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, 1));
            // the row's exponent: slot i mod 4, once the consumers of tile i - 4 have read it
            const int q = i % kSe64;
            if (i >= kSe64 && !mbar_wait_warp(&bar_se[q], (uint32_t)(((i - kSe64) / kSe64) & 1))) {
                *vfailed = 1;
                break;
            }
            if (h == 0) rowexp[q][r] = emax;
            mbar_arrive(&bar_sf[q]);
            // A buffer b: the MMAs of tile i - 2 must be done reading it
            if (i >= 2 && !mbar_wait_warp(&bar_d[b], (uint32_t)(((i - 2) >> 1) & 1))) {
                *vfailed = 1;
                break;
            }
            tc_fence_after();
            unsigned char *ab = abuf + (size_t)b * kPlanes * kAPlaneB + arow;
            // an FP16 pair (1024 + b_re, 1024 + b_im) has the exponent byte 0x64 above
            // each offset digit b = d + 128 (0..256); times the sign s of the
            // component, plus -1152 s, it is s d exactly (one HFMA2)
            constexpr uint32_t kE = 0x64646464u;
            const uint32_t kOne = 0x3C003C00u, kNegBias = 0xE480E480u;   // (1, 1), (-1152, -1152)
#pragma unroll
            for (int g = 0; g < DH / 4; ++g) {
                // complex columns 4 g4 .. 4 g4 + 3 = K-elements 8 g4 .. 8 g4 + 7: one 16-byte core-matrix row per plane
                const int g4 = (DH / 4) * h + g;
                uint32_t w[kPlanes][4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const double2 x = v[4 * g + j];
                    const uint32_t xrh = (uint32_t)__double2hiint(x.x), xih = (uint32_t)__double2hiint(x.y);
                    const uint64_t tr = fixed47m(xrh, (uint32_t)__double2loint(x.x), emax);
                    const uint64_t ti = fixed47m(xih, (uint32_t)__double2loint(x.y), emax);
                    const uint32_t rh = (uint32_t)(tr >> 32), rl = (uint32_t)tr;
                    const uint32_t ih = (uint32_t)(ti >> 32), il = (uint32_t)ti;
                    // signs: bit 15 from the real part, bit 31 from the imaginary part
                    const uint32_t sgn = __byte_perm(xrh, xih, 0x7030u) & 0x80008000u;
                    const uint32_t sig = kOne | sgn, bia = kNegBias ^ sgn;
                    // byte k of t + kDigitOff is digit 5 - k; pick each digit pair
                    // (re, im) next to the exponent bytes
                    const uint32_t p23 = __byte_perm(rl, il, 0x6723u), p45 = __byte_perm(rl, il, 0x4501u);
                    uint32_t q[kPlanes];
                    q[0] = 0x64006400u | (rh >> 8) | ((ih >> 8) << 16);
                    q[1] = __byte_perm(__byte_perm(rh, ih, 0x0400u), kE, 0x4240u);
                    q[2] = __byte_perm(p23, kE, 0x4240u);
                    q[3] = __byte_perm(p23, kE, 0x4341u);
                    q[4] = __byte_perm(p45, kE, 0x4240u);
                    q[5] = __byte_perm(p45, kE, 0x4341u);
#pragma unroll
                    for (int p = 0; p < kPlanes; ++p) {
                        const __half2 hd = __hfma2(*reinterpret_cast<const __half2 *>(&q[p]),
                                                   *reinterpret_cast<const __half2 *>(&sig),
                                                   *reinterpret_cast<const __half2 *>(&bia));
                        w[p][j] = *reinterpret_cast<const uint32_t *>(&hd);
                    }
                }
#pragma unroll
                for (int p = 0; p < kPlanes; ++p)
                    *reinterpret_cast<uint4 *>(ab + (size_t)p * kAPlaneB + ((uint32_t)g4 << 7)) =
                        make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
            }
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(&bar_a[b]);
        }
    } else if (warp < 16) {
        // consumers: warp w may read TMEM lanes 32 (w mod 4) .. + 31 (rows of the
        // tile); warps 8-11 take columns 0..15 of every level, warps 12-15 16..31
        const int quarter = warp & 3, half = (warp - 8) >> 2;
        const int r = 32 * quarter + lane;
        uint32_t ur;
        uint64_t gr;
        row_offsets(r, ur, gr);
        for (int i = 0; i < iters && !warp_flag(vfailed); ++i) {
            const int b = i & 1;
            const uint64_t base = tile_base(blockIdx.x + (uint64_t)i * step) | gr;
            if (!mbar_wait_warp(&bar_d[b], (uint32_t)((i >> 1) & 1))) {
                *vfailed = 1;
                break;
            }
            const int q = i % kSe64;
            if (!mbar_wait_warp(&bar_sf[q], (uint32_t)((i / kSe64) & 1))) {
                *vfailed = 1;
                break;
            }
            const int er = (int)rowexp[q][r];
            mbar_arrive(&bar_se[q]);
            tc_fence_after();
            const uint32_t lb = taddr + ACC * (uint32_t)b + ((uint32_t)(quarter * 32) << 16);
            // chunks of 4 columns (two complex outputs); the loads of chunk c + 1
            // are issued before chunk c is converted, so their latency overlaps it
            constexpr int CW = 4, NCH = (K / 2) / CW;
            const int nb = half * (K / 2);
            uint32_t d[2][kPlanes][CW];
#pragma unroll
            for (int l = 0; l < kPlanes; ++l) tmem_ld4_nowait(lb + 32u * (uint32_t)l + (uint32_t)nb, d[0][l]);
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                uint32_t (&dc)[kPlanes][CW] = d[c & 1];
                tmem_wait_ld_regs(dc);
                if (c + 1 < NCH) {
#pragma unroll
                    for (int l = 0; l < kPlanes; ++l)
                        tmem_ld4_nowait(lb + 32u * (uint32_t)l + (uint32_t)(nb + CW * (c + 1)), d[(c + 1) & 1][l]);
                }
                const int n0 = nb + CW * c;
                double o[CW];
#pragma unroll
                for (int e = 0; e < CW; ++e) {
                    // exact integers below 2^22: the FP32 bits of D + 1.5 2^23 are
                    // kMagic + D, so pairs combine on the raw bits (mod 2^32) and
                    // one constant removes the magic: D_0 256 + D_1 = u_0 256 + u_1 - 257 kMagic
                    constexpr uint32_t kMagic = 0x4B400000u;
                    uint32_t u[kPlanes];
#pragma unroll
                    for (int l = 0; l < kPlanes; ++l) u[l] = __float_as_uint(__uint_as_float(dc[l][e]) + 12582912.0f);
                    const int32_t a01 = (int32_t)(u[0] * 256u + u[1] - 257u * kMagic);
                    const int32_t a23 = (int32_t)(u[2] * 256u + u[3] - 257u * kMagic);
                    const int32_t a45 = (int32_t)(u[4] * 256u + u[5] - 257u * kMagic);
                    // T = sum_l D_l 256^(5 - l), |T| < 2^63
                    const long long T = (long long)a01 * (1ll << 32) + (long long)a23 * 65536 + (long long)a45;
                    // T 2^(E_r + F_n - 54), E = biased exponent - 1022: T as an FP64
                    // value (rounded to nearest above 2^53), the scale added to its
                    // exponent field; zero, and results below the normal range, give 0
                    const double f = __ll2double_rn(T);
                    const int fh = __double2hiint(f);
                    const int ef = (fh >> 20) & 0x7FF;
                    const int sc = er + colexp[n0 + e] - 2044 - 54;
                    o[e] = (ef != 0 && ef + sc > 0) ? __hiloint2double(fh + sc * (1 << 20), __double2loint(f)) : 0.0;
                }
                // columns n0 .. n0 + 3 = complex columns n0 / 2, n0 / 2 + 1
#pragma unroll
                for (int cc = 0; cc < CW / 2; ++cc)
                    *reinterpret_cast<double2 *>(st + 2 * (base | gc[n0 / 2 + cc])) = make_double2(o[2 * cc], o[2 * cc + 1]);
            }
            tc_fence_before();
            mbar_arrive(&bar_e[b]);
        }
    } else if (warp == 16 && lane == 0) {
        // issuer: digit plane p of A against W planes 0 .. 5 - p, into levels p .. 5
        const uint32_t sw = smem_u32(wsm);
        const uint32_t sa = smem_u32(abuf);
        int nd = 0;
        for (int i = 0; i < iters && !*vfailed; ++i) {
            const int b = i & 1;
            if (!mbar_wait_bounded(&bar_a[b], (uint32_t)((i >> 1) & 1))) { *vfailed = 1; break; }
            if (i >= 2 && !mbar_wait_bounded(&bar_e[b], (uint32_t)(((i - 2) >> 1) & 1))) { *vfailed = 1; break; }
            tc_fence_after();
            const uint32_t d0 = taddr + ACC * (uint32_t)b;
            const uint32_t a0 = sa + (uint32_t)b * kPlanes * kAPlaneB;
#pragma unroll 1
            for (int p = 0; p < kPlanes; ++p) {
                const uint32_t idesc = make_idesc_f16(kRows64, (kPlanes - p) * K);
#pragma unroll
                for (int ks = 0; ks < K / 16; ++ks)
                    mma_f16_ss(d0 + 32u * (uint32_t)p, make_desc(a0 + (uint32_t)p * kAPlaneB + 256u * ks, 128, SBO),
                               make_desc(sw + 256u * ks, 128, SBO), idesc, (p | ks) != 0);
            }
            mma_commit(&bar_d[b]);
            nd = i + 1;
        }
        if (*vfailed && nd > 0) mbar_wait_bounded(&bar_d[(nd - 1) & 1], (uint32_t)(((nd - 1) >> 1) & 1));
    }
    __syncthreads();
    if (tid == 0 && *vfailed) atomicExch(status, SIM_ETIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, NCOLS);
}

constexpr size_t c128_smem_bytes()
{
    return kStage64 * (size_t)kTAmp64 * 16 + 2 * (size_t)kPlanes * kAPlaneB + (size_t)kPlanes * kPlaneB;
}

}  // namespace

size_t fused_c128_slot_bytes() { return kSlot64; }

int fused_c128_prepare(qsim_state *s, int *grid)
{
    const size_t smem = c128_smem_bytes();
    if (cudaFuncSetAttribute((const void *)k_fused_c128, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute((const void *)k_fused_c128, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "complex128 fused kernel attributes");
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_fused_c128, kT64Threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return fail(SIM_ECUDA, "fused apply: the complex128 kernel does not fit on an SM");
    const uint64_t tiles = (1ull << s->n) / kTAmp64;
    *grid = (int)std::min<uint64_t>(tiles, (uint64_t)s->num_sms);
    return SIM_OK;
}

int launch_fuse_build_c128(qsim_state *s, const void *gates, const int *goff, int nb, void *out)
{
    static_assert(sizeof(FGate64) == 72, "block gate layout");
    launch_begin(s, KC_FUSE_BUILD, (double)nb * kSlot64);
    k_fuse_build64<<<(unsigned)nb, 256, 0, s->stream>>>((const FGate64 *)gates, goff, (unsigned char *)out);
    return launch_end(s, "complex128 fused build");
}

int launch_fused_c128(qsim_state *s, const void *block, const int *pos, int grid)
{
    Apply64 a{};
    for (int i = 0; i < kQ64; ++i) a.pos[i] = pos[i];
    const uint64_t tiles = (1ull << s->n) / kTAmp64;
    // tensor-core work: 14 MMAs of 128 x 16 x (7 - p) 32 per tile
    const double flops = (double)tiles * 2.0 * kRows64 * 16.0 * 32.0 * 2.0 * (7 + 6 + 5 + 4 + 3 + 2 + 1);
    launch_begin(s, KC_FUSED_C128, 2.0 * (double)s->bytes, flops);
    k_fused_c128<<<(unsigned)grid, kT64Threads, c128_smem_bytes(), s->stream>>>((double *)s->amps,
                                                                                 (const unsigned char *)block, a,
                                                                                 tiles, s->dev_status);
    return launch_end(s, "complex128 fused apply");
}

}  // namespace qsim
