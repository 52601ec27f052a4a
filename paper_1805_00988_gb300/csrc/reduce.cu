// reduce.cu -- state initialisation, probabilities, FP64 reductions,
// single-qubit collapse and shot sampling.
//
// Probabilities are |a_j|^2 (App. B.3).  Every sum of probabilities (norm,
// the two halves of a single-qubit measurement, <sum Z>, the sampling CDF) is
// accumulated in FP64 over a fixed grid and a fixed tree, so results are
// bit-reproducible run to run.  complex128 squares are FP64 FMAs; complex64
// squares are exact FP32 products summed with compensation in short chunks
// that are carried into FP64 (see "compensated FP32 sums of squares").
//
// Sampling (§2.4: many outcomes from one state without re-running the gates)
// is an inverse CDF over the FP64 prefix of |a_j|^2 that is never
// materialised for the whole state: sums per sub-block of 256 amplitudes and
// per block of 32 sub-blocks (one read of the state), one scan over the block
// sums, shots bucketed by block (counting sort), then per shot one warp picks
// the sub-block from the block's sub-sums and scans only those 256
// amplitudes (2 KB of complex64 per shot instead of the whole block).
#include <cmath>

#include "internal.cuh"

namespace qsim {

namespace {

// ---------------------------------------------------------------- SplitMix64
// Steele, Lea & Flood, OOPSLA 2014: add the golden gamma, then the variant-13
// finaliser.  Uniform draw u = (x >> 11) * 2^-53.
__host__ __device__ __forceinline__ uint64_t smix(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
__host__ __device__ __forceinline__ double unif(uint64_t seed, uint64_t s)
{
    return (double)(smix(seed + s) >> 11) * 0x1.0p-53;
}

// ---------------------------------------------------------------- init
// Zero the state with 16-byte stores and write amplitude j = 1.
__global__ void k_init_basis(uint4 *__restrict__ st, uint64_t nvec, uint64_t jvec, uint4 jval)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec;
         i += (uint64_t)gridDim.x * blockDim.x)
        st[i] = (i == jvec) ? jval : make_uint4(0, 0, 0, 0);
}

// ---------------------------------------------------------------- block reduce
template <int NT>
__device__ __forceinline__ void block_sum2(double &a, double &b, double *sh)
{
    // fixed-order tree: warp butterflies, then warp 0 over the warp results
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[2 * w] = a; sh[2 * w + 1] = b; }
    __syncthreads();
    if (w == 0) {
        a = (l < NT / 32) ? sh[2 * l] : 0.0;
        b = (l < NT / 32) ? sh[2 * l + 1] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
    }
    __syncthreads();
}

template <typename R>
__device__ __forceinline__ double sq(R re, R im)
{
    const double r = (double)re, i = (double)im;
    return fma(r, r, i * i);
}

// FP32 -> FP64 with integer operations (the FP64 pipe of this GPU is narrow,
// so the conversion would cost as much as the arithmetic): a normal float is
// widened exactly by rebiasing the exponent (127 -> 1023) and shifting the
// mantissa; zero and subnormals become 0 (their squares are below 1e-76 and
// do not change an FP64 sum of probabilities); states hold no inf / NaN.
__device__ __forceinline__ double widen(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint64_t d = ((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                       ((uint64_t)(u & 0x007FFFFFu) << 29);
    return e ? __longlong_as_double((long long)d) : 0.0;
}

template <>
__device__ __forceinline__ double sq<float>(float re, float im)
{
    const double r = widen(re), i = widen(im);
    return fma(r, r, i * i);
}


// a += |re + i im|^2 as two FP64 FMAs (both squares exact in FP64 for a
// complex64 amplitude)
template <typename R>
__device__ __forceinline__ void acc_sq(double &a, R re, R im)
{
    const double r = (double)re, i = (double)im;
    a = fma(r, r, a);
    a = fma(i, i, a);
}
template <>
__device__ __forceinline__ void acc_sq<float>(double &a, float re, float im)
{
    const double r = widen(re), i = widen(im);
    a = fma(r, r, a);
    a = fma(i, i, a);
}

// ---------------------------------------------------------------- compensated FP32 sums of squares
// The FP64 pipe of this GPU runs at about 1/64 of the FP32 rate, so two FP64
// FMAs per complex64 amplitude make a sum of |a|^2 FP64-bound, at about 2.7x
// the time it takes to read the state.  The complex64 reductions therefore
// take their squares and partial sums with error-free FP32 transformations and
// carry them into FP64 once per 8 amplitudes (16 squares):
//  * a chunk is rescaled by an exact power of two 2^(127 - k), k the exponent
//    of its largest component, so that no square overflows or is lost to
//    underflow (the scaling is undone exactly in the FP64 exponent);
//  * x^2 = h + l exactly, with h = fl(x * x) and l = fma(x, x, -h) (Dekker's
//    product, formed with an FMA); h enters the running sum s through Knuth's
//    TwoSum (s + h = t + err exactly), and err + l accumulate in e: the Dot2
//    scheme of Ogita, Rump & Oishi (SIAM J. Sci. Comput. 26(6), 2005);
//  * for m non-negative terms |(s + e) - sum| <= (m + 1)^2 u^2 sum (u = 2^-24,
//    m = 16: about 1e-12 relative in the worst case, where every rounding
//    error takes its maximum with the same sign; around 1e-15 in practice);
//  * s and e widen to FP64 exactly.
// The __f*_rn intrinsics keep the compiler from contracting a product and a
// sum into one FMA, which would break the exactness of the transformations.
struct Sq32 {
    float s = 0.f, e = 0.f;                  // value = s + e
    __device__ __forceinline__ void two_sum(float h)
    {
        const float t = __fadd_rn(s, h);
        const float z = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(h, z));
        s = t;
        e = __fadd_rn(e, err);
    }
    // += x^2
    __device__ __forceinline__ void add_sq(float x)
    {
        const float h = __fmul_rn(x, x);
        const float l = __fmaf_rn(x, x, -h);
        const float t = __fadd_rn(s, h);
        const float z = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(h, z));
        s = t;
        e = __fadd_rn(e, __fadd_rn(err, l));
    }
    // += x * w (w a small integer; the product is split exactly like a square)
    __device__ __forceinline__ void add_prod(float x, float w)
    {
        const float h = __fmul_rn(x, w);
        const float l = __fmaf_rn(x, w, -h);
        two_sum(h);
        e = __fadd_rn(e, l);
    }
};

// Exact power-of-two rescaling of a chunk.  amax = the largest |component|;
// k = its biased exponent clamped to [1, 253], so 2^(127 - k) is a normal float
// and the largest scaled component lies in [1, 2) (k = 1 covers zero and
// subnormal chunks).  Squares of the scaled chunk are the true squares times
// 2^-sh, with sh = 2 (k - 127).
struct Pow2 {
    float scale;
    int sh;
};
__device__ __forceinline__ Pow2 pow2_for(float amax)
{
    const int k = min(max((int)(__float_as_uint(amax) >> 23), 1), 253);
    return {__uint_as_float((uint32_t)(254 - k) << 23), 2 * (k - 127)};
}
__device__ __forceinline__ float absmax4(float m, const float4 &v)
{
    return fmaxf(fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y))), fmaxf(fabsf(v.z), fabsf(v.w)));
}
__device__ __forceinline__ float4 scale4(const float4 &v, float c)
{
    return make_float4(__fmul_rn(v.x, c), __fmul_rn(v.y, c), __fmul_rn(v.z, c), __fmul_rn(v.w, c));
}

// f * 2^sh as an FP64, exactly, by integer operations on the exponent field
// (|sh| <= 252 and f a partial sum of a rescaled chunk, so the FP64 exponent
// stays in range); zero and subnormal f give 0.
__device__ __forceinline__ double widen_pow2(float f, int sh)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    const int ex = (int)e + 896 + sh;
    const uint64_t d = ((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)ex << 52) |
                       ((uint64_t)(u & 0x007FFFFFu) << 29);
    return e ? __longlong_as_double((long long)d) : 0.0;
}
__device__ __forceinline__ double widen_sum(const Sq32 &a, int sh)
{
    return widen_pow2(a.s, sh) + widen_pow2(a.e, sh);
}

// VEC amplitudes per 16-byte vector: 2 for complex64, 1 for complex128.
// raw() issues the load only; sq2() turns it into |a|^2 in FP64.  Callers
// issue a batch of raw loads before any arithmetic so that each thread keeps
// several 16-byte requests in flight.
template <typename R> struct AV;
template <> struct AV<float> {
    static constexpr int VEC = 2;
    using Raw = float4;
    __device__ __forceinline__ static Raw raw(const float *st, uint64_t v) { return reinterpret_cast<const float4 *>(st)[v]; }
    __device__ __forceinline__ static void sq2(const Raw &x, double p[2])
    {
        p[0] = sq<float>(x.x, x.y);
        p[1] = sq<float>(x.z, x.w);
    }
    __device__ __forceinline__ static void load(const float *st, uint64_t v, double p[2]) { sq2(raw(st, v), p); }
    __device__ __forceinline__ static void parts(const Raw &x, float re[2], float im[2])
    {
        re[0] = x.x; im[0] = x.y; re[1] = x.z; im[1] = x.w;
    }
};
template <> struct AV<double> {
    static constexpr int VEC = 1;
    using Raw = double2;
    __device__ __forceinline__ static Raw raw(const double *st, uint64_t v) { return reinterpret_cast<const double2 *>(st)[v]; }
    __device__ __forceinline__ static void sq2(const Raw &x, double p[2])
    {
        p[0] = sq<double>(x.x, x.y);
        p[1] = 0.0;
    }
    __device__ __forceinline__ static void load(const double *st, uint64_t v, double p[2]) { sq2(raw(st, v), p); }
    __device__ __forceinline__ static void parts(const Raw &x, double re[1], double im[1])
    {
        re[0] = x.x; im[0] = x.y;
    }
};

// one amplitude as a vector type
template <typename R> struct Amp;
template <> struct Amp<float> { using T = float2; };
template <> struct Amp<double> { using T = double2; };

constexpr int kBatch = 8;     // 16-byte loads in flight per thread

// Masked FP64 sums over a contiguous range per block.
//   RED_NORM: out0 = sum |a|^2                    (two FP64 FMAs per amplitude)
//   RED_BIT : out0 = sum over bit q = 0, out1 = sum over bit q = 1
//   RED_EXPZ: out0 = sum |a_x|^2 (n - 2 popcount x)  (weights from a table),
//             out1 = sum |a|^2 (the norm, from the same pass)
template <typename R, int MODE>
__global__ void __launch_bounds__(kRedThreads) k_masked_sum(const R *__restrict__ st, uint64_t nvec, uint64_t per,
                                                            int q, int n, double *__restrict__ partial)
{
    constexpr int VEC = AV<R>::VEC;
    __shared__ double sh[2 * kRedThreads / 32];
    __shared__ double wtab[64];                 // RED_EXPZ: wtab[k] = n - 2k
    if (MODE == RED_EXPZ) {
        for (int k = threadIdx.x; k <= n; k += kRedThreads) wtab[k] = (double)(n - 2 * k);
        __syncthreads();
    }
    const uint64_t lo = (uint64_t)blockIdx.x * per;
    const uint64_t hi = min(nvec, lo + per);
    double a = 0.0, b = 0.0;
    auto add = [&](uint64_t v, const typename AV<R>::Raw &x) {
        R re[VEC], im[VEC];
        AV<R>::parts(x, re, im);
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            const uint64_t i = v * VEC + e;
            if (MODE == RED_NORM) {
                acc_sq<R>(a, re[e], im[e]);
            } else if (MODE == RED_BIT) {
                if ((i >> q) & 1ull) acc_sq<R>(b, re[e], im[e]);
                else acc_sq<R>(a, re[e], im[e]);
            } else {
                const double p2 = sq<R>(re[e], im[e]);
                a = fma(p2, wtab[__popcll(i)], a);
                b += p2;
            }
        }
    };
    uint64_t v = lo + threadIdx.x;
    for (; v + (uint64_t)(kBatch - 1) * kRedThreads < hi; v += (uint64_t)kBatch * kRedThreads) {
        typename AV<R>::Raw x[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) x[u] = AV<R>::raw(st, v + (uint64_t)u * kRedThreads);
#pragma unroll
        for (int u = 0; u < kBatch; ++u) add(v + (uint64_t)u * kRedThreads, x[u]);
    }
    for (; v < hi; v += kRedThreads) add(v, AV<R>::raw(st, v));
    block_sum2<kRedThreads>(a, b, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

// complex64 norm (MODE RED_NORM) and the two halves of qubit q (RED_BIT) with
// the compensated FP32 sums above: per batch of 8 16-byte vectors (16
// amplitudes) one power-of-two scale, two carries into FP64 (8 amplitudes
// each).  The batches, the grid and the FP64 tree are those of k_masked_sum.
template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_sum_sq32(const float *__restrict__ st, uint64_t nvec, uint64_t per,
                                                          int q, double *__restrict__ partial)
{
    static_assert(MODE == RED_NORM || MODE == RED_BIT, "norm or one qubit's halves");
    __shared__ double sh[2 * kRedThreads / 32];
    const uint64_t lo = (uint64_t)blockIdx.x * per;
    const uint64_t hi = min(nvec, lo + per);
    const float4 *st4 = reinterpret_cast<const float4 *>(st);
    double a = 0.0, b = 0.0;
    // the amplitudes of vector v (indices 2v, 2v + 1) go to A (bit q = 0) or B
    auto add_vec = [&](Sq32 &A, Sq32 &B, uint64_t v, const float4 &y) {
        if (MODE == RED_NORM) {
            A.add_sq(y.x); A.add_sq(y.y); A.add_sq(y.z); A.add_sq(y.w);
        } else {
            const bool b0 = ((2 * v) >> q) & 1ull, b1 = ((2 * v + 1) >> q) & 1ull;
            Sq32 c = b0 ? B : A;
            c.add_sq(y.x); c.add_sq(y.y);
            if (b0) B = c; else A = c;
            c = b1 ? B : A;
            c.add_sq(y.z); c.add_sq(y.w);
            if (b1) B = c; else A = c;
        }
    };
    uint64_t v = lo + threadIdx.x;
    for (; v + (uint64_t)(kBatch - 1) * kRedThreads < hi; v += (uint64_t)kBatch * kRedThreads) {
        float4 x[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) x[u] = st4[v + (uint64_t)u * kRedThreads];
        float m = 0.f;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) m = absmax4(m, x[u]);
        const Pow2 p = pow2_for(m);
#pragma unroll
        for (int h = 0; h < kBatch; h += 4) {
            Sq32 A, B;
#pragma unroll
            for (int u = h; u < h + 4; ++u) add_vec(A, B, v + (uint64_t)u * kRedThreads, scale4(x[u], p.scale));
            a += widen_sum(A, p.sh);
            if (MODE == RED_BIT) b += widen_sum(B, p.sh);
        }
    }
    for (; v < hi; v += kRedThreads) {
        const float4 x = st4[v];
        const Pow2 p = pow2_for(absmax4(0.f, x));
        Sq32 A, B;
        add_vec(A, B, v, scale4(x, p.scale));
        a += widen_sum(A, p.sh);
        if (MODE == RED_BIT) b += widen_sum(B, p.sh);
    }
    block_sum2<kRedThreads>(a, b, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

// <sum Z> over chunks of 16 consecutive amplitudes (n >= 4): for x = 16 ch +
// e, popcount(x) = popcount(ch) + popcount(e), so a thread sums the squares of
// a chunk into five bins by popcount(e) (two FP64 FMAs per amplitude, e known
// at compile time) and adds bin j with weight n - 2 (popcount(ch) + j): five
// FMAs per 16 amplitudes instead of one weighted FMA each.  The second
// partial is the norm (the bins' sum) from the same pass.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_expz_chunks(const R *__restrict__ st, uint64_t nch, uint64_t per,
                                                             int n, double *__restrict__ partial)
{
    using T = typename Amp<R>::T;
    __shared__ double sh[2 * kRedThreads / 32];
    __shared__ double wtab[64];                  // wtab[k] = n - 2k
    for (int k = threadIdx.x; k <= n; k += kRedThreads) wtab[k] = (double)(n - 2 * k);
    __syncthreads();
    const uint64_t lo = (uint64_t)blockIdx.x * per;
    const uint64_t hi = min(nch, lo + per);
    double a = 0.0, b = 0.0;
    for (uint64_t ch = lo + threadIdx.x; ch < hi; ch += kRedThreads) {
        double bin[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        if (sizeof(R) == 4) {
            const float4 *q = reinterpret_cast<const float4 *>(st) + ch * 8;
            float4 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = q[u];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                acc_sq<float>(bin[__builtin_popcount(2 * u)], x[u].x, x[u].y);
                acc_sq<float>(bin[__builtin_popcount(2 * u + 1)], x[u].z, x[u].w);
            }
        } else {
            const T *q = reinterpret_cast<const T *>(st) + ch * 16;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                T x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) x[u] = q[8 * h + u];
#pragma unroll
                for (int u = 0; u < 8; ++u) acc_sq<R>(bin[__builtin_popcount(8 * h + u)], x[u].x, x[u].y);
            }
        }
        const int pc = __popcll(ch);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            a = fma(wtab[pc + j], bin[j], a);
            b += bin[j];
        }
    }
    block_sum2<kRedThreads>(a, b, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

// complex64 <sum Z> over chunks of 16 consecutive amplitudes (n >= 4): the
// same popcount bins as k_expz_chunks, each a compensated FP32 sum of squares
// of the chunk rescaled by one power of two; the bins are weighted by the
// integers n - 2 (popcount(ch) + j) with exact FP32 products into one
// compensated sum, carried into FP64 once per chunk.  Bins hold at most 12
// squares; the weighted sum cancels, so its error is relative to
// sum_j |w_j| bin_j <= n * (the chunk's sum of squares).  The second
// partial is the norm: the bins' compensated sum, carried into FP64 per chunk.
__global__ void __launch_bounds__(kRedThreads) k_expz32(const float *__restrict__ st, uint64_t nch, uint64_t per,
                                                        int n, double *__restrict__ partial)
{
    __shared__ double sh[2 * kRedThreads / 32];
    const uint64_t lo = (uint64_t)blockIdx.x * per;
    const uint64_t hi = min(nch, lo + per);
    const float4 *st4 = reinterpret_cast<const float4 *>(st);
    double a = 0.0, b = 0.0;
    for (uint64_t ch = lo + threadIdx.x; ch < hi; ch += kRedThreads) {
        float4 x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = st4[ch * 8 + u];
        float m = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) m = absmax4(m, x[u]);
        const Pow2 p = pow2_for(m);
        Sq32 bin[5];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float4 y = scale4(x[u], p.scale);
            bin[__builtin_popcount(2 * u)].add_sq(y.x);
            bin[__builtin_popcount(2 * u)].add_sq(y.y);
            bin[__builtin_popcount(2 * u + 1)].add_sq(y.z);
            bin[__builtin_popcount(2 * u + 1)].add_sq(y.w);
        }
        const int pc = __popcll(ch);
        Sq32 w, t;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const float wj = (float)(n - 2 * (pc + j));
            w.add_prod(bin[j].s, wj);
            w.e = __fmaf_rn(bin[j].e, wj, w.e);
            t.two_sum(bin[j].s);
            t.e = __fadd_rn(t.e, bin[j].e);
        }
        a += widen_sum(w, p.sh);
        b += widen_sum(t, p.sh);
    }
    block_sum2<kRedThreads>(a, b, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

__global__ void __launch_bounds__(kRedThreads) k_final_sum(const double *__restrict__ partial, int nblk,
                                                           double *__restrict__ out)
{
    __shared__ double sh[2 * kRedThreads / 32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblk; i += kRedThreads) {
        a += partial[2 * i];
        b += partial[2 * i + 1];
    }
    block_sum2<kRedThreads>(a, b, sh);
    if (threadIdx.x == 0) { out[0] = a; out[1] = b; }
}

// ---------------------------------------------------------------- probabilities
template <typename R, typename O>
__global__ void k_probabilities(const R *__restrict__ st, uint64_t N, O *__restrict__ p)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const R re = st[2 * i], im = st[2 * i + 1];
        if (sizeof(O) == sizeof(R)) p[i] = (O)(re * re + im * im);
        else p[i] = (O)sq<R>(re, im);
    }
}

// ---------------------------------------------------------------- collapse
template <typename R>
__global__ void k_collapse(R *__restrict__ st, uint64_t N, int q, int outcome, R scale)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if ((int)((i >> q) & 1ull) == outcome) {
            st[2 * i] *= scale;
            st[2 * i + 1] *= scale;
        } else {
            st[2 * i] = (R)0;
            st[2 * i + 1] = (R)0;
        }
    }
}

// ---------------------------------------------------------------- sampling
constexpr int kSampleLog = 13;             // 8192 amplitudes per sampling block
constexpr int kScanThreads = 1024;

// Sub-blocks: min(256, bs) amplitudes, nsub = bs / sub <= 32 per block; lane
// l of a warp takes amplitudes l*apl .. l*apl + apl - 1 of a sub-block
// (apl = max(1, sub / 32)), so a lane-serial prefix followed by a warp scan
// is the sub-block's prefix in index order.
constexpr int kSubLog = 8;

struct SubGeo {
    uint32_t sub, nsub, apl, lanes;
    __host__ __device__ explicit SubGeo(uint64_t bs)
    {
        sub = (uint32_t)(bs < (1ull << kSubLog) ? bs : (1ull << kSubLog));
        nsub = (uint32_t)(bs / sub);
        apl = sub >= 32 ? sub / 32 : 1;
        lanes = sub / apl;
    }
};


// FP64 |a|^2 of the apl amplitudes of lane `lane` in sub-block `j` (zeros for
// idle lanes and unused slots), loads first
template <typename R>
__device__ __forceinline__ void lane_squares(const R *st, uint64_t base, const SubGeo &g, uint32_t j, int lane,
                                             double p[8])
{
    using T = typename Amp<R>::T;
    const T *a = reinterpret_cast<const T *>(st) + base + (uint64_t)j * g.sub + (uint64_t)lane * g.apl;
    T x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e)
        if ((uint32_t)lane < g.lanes && (uint32_t)e < g.apl) x[e] = a[e];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        p[e] = 0.0;
        if ((uint32_t)lane < g.lanes && (uint32_t)e < g.apl) acc_sq<R>(p[e], x[e].x, x[e].y);
    }
}

// warp inclusive scan of lanes 0..31, fixed order (shfl_up doubling)
__device__ __forceinline__ double warp_incl_scan(double x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// One CTA (8 warps) per block of bs amplitudes.  Groups of 8 lanes own one
// sub-block each (4 per warp, 32 per CTA): lane g of a group accumulates a
// contiguous eighth of the sub-block (complex64 full sub-blocks: compensated
// FP32 squares carried into FP64 every 8 amplitudes; otherwise two FP64 FMAs
// per amplitude), and a 3-step xor tree inside the group gives the sub-sum.
// Warp 0 then scans the block's sub-sums (warp_incl_scan) and the block sum is
// the scan's last element -- k_resolve repeats that scan bit for bit.
// kZ (complex64 full sub-blocks only): the same pass also forms the block's
// <sum Z> partial as k_expz32 does (each 16-amplitude chunk's squares binned
// by the popcount of the local index, weighted by n - 2 popcount, one
// compensated sum carried into FP64), written to zpart[2 b] (zpart[2 b + 1] =
// 0, the pair layout k_final_sum reads).  The sub-sums are computed exactly as
// without it.
template <typename R, bool kZ = false>
__global__ void __launch_bounds__(256) k_sub_sums(const R *__restrict__ st, uint64_t bs, double *__restrict__ sub,
                                                  double *__restrict__ bsum, int n = 0,
                                                  double *__restrict__ zpart = nullptr)
{
    using T = typename Amp<R>::T;
    const SubGeo g(bs);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t j = (uint32_t)(warp * 4 + (lane >> 3));       // this group's sub-block
    const uint32_t gl = (uint32_t)(lane & 7);                    // lane within the group
    const uint64_t base = (uint64_t)blockIdx.x * bs;
    __shared__ double ss[32];
    __shared__ double zs[8];
    double t = 0.0, z = 0.0;
    if (j < g.nsub) {
        const uint32_t per = g.sub >= 8 ? g.sub / 8 : 1;         // amplitudes per lane
        if (gl * per < g.sub) {
            const T *a = reinterpret_cast<const T *>(st) + base + (uint64_t)j * g.sub + (uint64_t)gl * per;
            if (sizeof(R) == 4 && per == 32) {
                // complex64, full sub-block: 16 aligned 16-byte loads per lane,
                // 8 in flight; compensated FP32 squares, one scale per 16
                // amplitudes, carried into FP64 every 8
                const float4 *a4 = reinterpret_cast<const float4 *>(a);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float4 x[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) x[u] = a4[h * 8 + u];
                    float m = 0.f;
#pragma unroll
                    for (int u = 0; u < 8; ++u) m = absmax4(m, x[u]);
                    const Pow2 pw = pow2_for(m);
#pragma unroll
                    for (int c = 0; c < 8; c += 4) {
                        Sq32 A;
#pragma unroll
                        for (int u = c; u < c + 4; ++u) {
                            const float4 y = scale4(x[u], pw.scale);
                            A.add_sq(y.x); A.add_sq(y.y); A.add_sq(y.z); A.add_sq(y.w);
                        }
                        t += widen_sum(A, pw.sh);
                    }
                    if constexpr (kZ) {
                        // amplitudes 16 ch .. 16 ch + 15: x[u] holds local indices 2u, 2u + 1
                        const uint64_t ch = ((base + (uint64_t)j * g.sub + (uint64_t)gl * per) >> 4) + (uint64_t)h;
                        Sq32 bin[5];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float4 y = scale4(x[u], pw.scale);
                            bin[__builtin_popcount(2 * u)].add_sq(y.x);
                            bin[__builtin_popcount(2 * u)].add_sq(y.y);
                            bin[__builtin_popcount(2 * u + 1)].add_sq(y.z);
                            bin[__builtin_popcount(2 * u + 1)].add_sq(y.w);
                        }
                        const int pc = __popcll(ch);
                        Sq32 w;
#pragma unroll
                        for (int b = 0; b < 5; ++b) {
                            const float wb = (float)(n - 2 * (pc + b));
                            w.add_prod(bin[b].s, wb);
                            w.e = __fmaf_rn(bin[b].e, wb, w.e);
                        }
                        z += widen_sum(w, pw.sh);
                    }
                }
            } else {
                for (uint32_t e0 = 0; e0 < per; e0 += 8) {
                    T x[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (e0 + u < per) x[u] = a[e0 + u];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (e0 + u < per) acc_sq<R>(t, x[u].x, x[u].y);
                }
            }
        }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (gl == 0 && j < g.nsub) {
        ss[j] = t;
        sub[(uint64_t)blockIdx.x * g.nsub + j] = t;
    }
    if constexpr (kZ) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        if (lane == 0) zs[warp] = z;
    }
    __syncthreads();
    if (warp == 0) {
        const double c = warp_incl_scan(((uint32_t)lane < g.nsub) ? ss[lane] : 0.0, lane);
        if ((uint32_t)lane == g.nsub - 1) bsum[blockIdx.x] = c;
    }
    if constexpr (kZ) {
        if (threadIdx.x == 0) {
            double zz = 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w) zz += zs[w];
            zpart[2 * blockIdx.x] = zz;
            zpart[2 * blockIdx.x + 1] = 0.0;
        }
    }
}

// Exclusive scan of nb values in one CTA: contiguous segments per thread,
// serial inside a segment, a fixed Hillis-Steele scan over segment totals.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_exclusive(const T *__restrict__ in, T *__restrict__ out,
                                                                 uint64_t nb, T *__restrict__ total)
{
    __shared__ T seg[kScanThreads];
    const uint64_t per = (nb + kScanThreads - 1) / kScanThreads;
    const uint64_t lo = (uint64_t)threadIdx.x * per;
    const uint64_t hi = min(nb, lo + per);
    T loc = 0;
    for (uint64_t i = lo; i < hi; ++i) loc += in[i];
    seg[threadIdx.x] = loc;
    __syncthreads();
    for (int off = 1; off < kScanThreads; off <<= 1) {
        T v = (threadIdx.x >= (unsigned)off) ? seg[threadIdx.x - off] : (T)0;
        __syncthreads();
        seg[threadIdx.x] += v;
        __syncthreads();
    }
    T run = (threadIdx.x > 0) ? seg[threadIdx.x - 1] : (T)0;
    if (threadIdx.x == kScanThreads - 1) *total = seg[kScanThreads - 1];
    T acc = 0;
    for (uint64_t i = lo; i < hi; ++i) {
        out[i] = run + acc;
        acc += in[i];
    }
}

// Exclusive scan over many CTAs (the sampler's block sums are FP64, and one
// CTA adding 2^17 of them ran into the narrow FP64 pipe of a single SM):
// chunks of kScanChunk values, four contiguous values per thread.  Pass 1
// writes each chunk's total, the one-CTA scan above turns the totals into
// chunk offsets (and the grand total), pass 2 repeats the chunk's local scan
// (the same operations, so the same bits) and adds the chunk's offset.
constexpr int kScanChunk = 1024;

template <typename T>
__device__ __forceinline__ T chunk_local_scan(const T *__restrict__ in, uint64_t nb, T *sh, T &total, T v[4],
                                              uint64_t &lo)
{
    lo = (uint64_t)blockIdx.x * kScanChunk + 4u * threadIdx.x;
    T loc = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        v[e] = (lo + e < nb) ? in[lo + e] : (T)0;
        loc += v[e];
    }
    sh[threadIdx.x] = loc;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        const T y = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : (T)0;
        __syncthreads();
        sh[threadIdx.x] += y;
        __syncthreads();
    }
    total = sh[255];
    return (threadIdx.x > 0) ? sh[threadIdx.x - 1] : (T)0;
}

template <typename T>
__global__ void __launch_bounds__(256) k_scan_chunk_sums(const T *__restrict__ in, uint64_t nb, T *__restrict__ csum)
{
    __shared__ T sh[256];
    T v[4], total;
    uint64_t lo;
    chunk_local_scan<T>(in, nb, sh, total, v, lo);
    if (threadIdx.x == 0) csum[blockIdx.x] = total;
}

template <typename T>
__global__ void __launch_bounds__(256) k_scan_chunk_out(const T *__restrict__ in, uint64_t nb,
                                                        const T *__restrict__ cexcl, T *__restrict__ out)
{
    __shared__ T sh[256];
    T v[4], total;
    uint64_t lo;
    T run = chunk_local_scan<T>(in, nb, sh, total, v, lo) + cexcl[blockIdx.x];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (lo + e < nb) out[lo + e] = run;
        run += v[e];
    }
}

// shot s -> block: smallest b with bexcl[b] + bsum[b] > u_s * total; none ->
// the last block with a non-zero sum.
__global__ void k_locate(uint64_t shots, uint64_t seed, const double *__restrict__ bexcl,
                         const double *__restrict__ bsum, uint64_t nb, const double *__restrict__ total,
                         uint32_t *__restrict__ shot_blk, uint32_t *__restrict__ counts, uint64_t last_nz_blk)
{
    const double tot = *total;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const double t = unif(seed, s) * tot;
        uint64_t lo = 0, hi = nb;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (bexcl[mid] + bsum[mid] > t) hi = mid; else lo = mid + 1;
        }
        const uint32_t b = (uint32_t)((lo < nb) ? lo : last_nz_blk);
        shot_blk[s] = b;
        atomicAdd(&counts[b], 1u);
    }
}

// last block with a non-zero sum (single thread; nb scanned backwards)
__global__ void k_last_nonzero(const double *__restrict__ bsum, uint64_t nb, uint64_t *__restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        uint64_t b = nb;
        while (b > 0 && !(bsum[b - 1] > 0.0)) --b;
        *out = (b > 0) ? b - 1 : 0;
    }
}

__global__ void k_scatter(uint64_t shots, const uint32_t *__restrict__ shot_blk, uint32_t *__restrict__ cursor,
                          uint32_t *__restrict__ order)
{
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots;
         s += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t pos = atomicAdd(&cursor[shot_blk[s]], 1u);
        order[pos] = (uint32_t)s;
    }
}

// a power of two 2^d as a float for d <= 127; 0 below -126 (a lane that
// small against the largest one contributes nothing measurable)
__device__ __forceinline__ float pow2f(int d)
{
    return d < -126 ? 0.f : __uint_as_float((uint32_t)(127 + min(d, 127)) << 23);
}

// s + t as an unevaluated pair (hi, lo) (Knuth's TwoSum) added to (hi, lo)
__device__ __forceinline__ void df_add(float &hi, float &lo, float th, float tl)
{
    const float u = __fadd_rn(hi, th);
    const float z = __fsub_rn(u, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(u, z)), __fsub_rn(th, z));
    hi = u;
    lo = __fadd_rn(__fadd_rn(lo, tl), err);
}

// complex64, full sub-blocks (8 amplitudes per lane): lane `lane`'s part of
// the in-sub-block search.  The lane's prefix is kept as compensated FP32
// partial sums of its squares rescaled by a power of two (2^-sh, from the
// lane's largest component).  The lanes' totals are brought to one scale (the
// warp's largest sh) by exact powers of two and scanned across the warp as
// FP32 pairs (TwoSum), so the only FP64 work per shot is the target t - pre
// in that scale: this GPU's FP64 pipe runs at a small fraction of its FP32
// rate, and an FP64 warp scan per shot made the search FP64-bound.  The
// target relative to the lane's start, rescaled back to the lane's units, is
// compared with each partial sum as a float pair.  An amplitude that is
// exactly zero leaves the prefix unchanged and is never the first crossing.
// first = the first crossing in the lane (-1: none), last_nz = the last
// amplitude with non-zero probability (-1: none).  All 32 lanes call it.
__device__ __forceinline__ void lane_locate32(const float *st, uint64_t base, uint32_t j, int lane, double pre,
                                              double t, int &first, int &last_nz)
{
    const float4 *a4 =
        reinterpret_cast<const float4 *>(st) + (base + (uint64_t)j * (1u << kSubLog) + (uint64_t)lane * 8) / 2;
    float4 x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = a4[u];
    float m = 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u) m = absmax4(m, x[u]);
    const Pow2 pw = pow2_for(m);
    float cs[8], ce[8];
    bool nz[8];
    Sq32 A;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const float4 y = scale4(x[u], pw.scale);
        A.add_sq(y.x); A.add_sq(y.y);
        cs[2 * u] = A.s; ce[2 * u] = A.e;
        nz[2 * u] = x[u].x != 0.f || x[u].y != 0.f;
        A.add_sq(y.z); A.add_sq(y.w);
        cs[2 * u + 1] = A.s; ce[2 * u + 1] = A.e;
        nz[2 * u + 1] = x[u].z != 0.f || x[u].w != 0.f;
    }
    // the lane's total in the warp's common units 2^shm (shm >= pw.sh)
    const int shm = __reduce_max_sync(0xffffffffu, pw.sh);
    const float down = pow2f(pw.sh - shm);
    float ih = __fmul_rn(A.s, down), il = __fmul_rn(A.e, down);
    // inclusive warp scan of the pairs, then each lane's start = the previous
    // lane's inclusive sum
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float yh = __shfl_up_sync(0xffffffffu, ih, o);
        const float yl = __shfl_up_sync(0xffffffffu, il, o);
        if (lane >= o) df_add(ih, il, yh, yl);
    }
    float sh0 = __shfl_up_sync(0xffffffffu, ih, 1), sl0 = __shfl_up_sync(0xffffffffu, il, 1);
    if (lane == 0) { sh0 = 0.f; sl0 = 0.f; }
    // target relative to the sub-block start in common units (FP64, then a
    // float pair), minus the lane's start, back in the lane's units
    double Tc = (t - pre) * __longlong_as_double((long long)((uint64_t)(1023 - shm) << 52));
    Tc = fmin(fmax(Tc, -0x1p100), 0x1p100);
    const float th = __double2float_rn(Tc);
    const float tl = __double2float_rn(Tc - (double)th);
    float rh = th, rl = tl;
    df_add(rh, rl, -sh0, -sl0);
    const float up = pow2f(shm - pw.sh);
    const bool far = shm - pw.sh > 127;            // the lane is negligible next to the largest
    rh = far ? (rh > 0.f ? INFINITY : -INFINITY) : __fmul_rn(rh, up);
    rl = far ? 0.f : __fmul_rn(rl, up);
    first = -1;
    last_nz = -1;
#pragma unroll
    for (int e = 7; e >= 0; --e) {
        if (nz[e] && __fadd_rn(__fsub_rn(cs[e], rh), __fsub_rn(ce[e], rl)) > 0.f) first = e;
        if (last_nz < 0 && nz[e]) last_nz = e;
    }
}

// Persistent warps over the shots in block order (the counting sort puts the
// shots of one block next to each other): warp w takes shots
// [w * per, (w + 1) * per) of `order`.  On entering a new block the warp
// rebuilds that block's inclusive scan of sub-sums P (lane j holds P[j]; the
// same operations as k_sub_sums, so the same bits) and its exclusive prefix.
// Per shot: t = u_s * total; the sub-block is the first j with
// bexcl + P[j] > t; the warp scans its amplitudes (lane-serial prefix, then a
// warp scan of lane totals) and the outcome is the first index whose prefix
// exceeds t.  Where rounding leaves no crossing (t within an ulp of a
// boundary), the last sub-block / amplitude with non-zero probability is
// taken.
template <typename R>
__global__ void __launch_bounds__(256) k_resolve(const R *__restrict__ st, uint64_t bs, uint64_t seed,
                                                 const double *__restrict__ bexcl, const double *__restrict__ total,
                                                 const double *__restrict__ sub, const uint32_t *__restrict__ shot_blk,
                                                 const uint32_t *__restrict__ order, uint64_t shots, uint64_t per,
                                                 uint64_t *__restrict__ out)
{
    const SubGeo g(bs);
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t k0 = warp * per;
    const uint64_t k1 = min(shots, k0 + per);
    const double tot = *total;
    uint32_t cur = 0xFFFFFFFFu;          // block whose scan the warp holds
    double Pl = 0.0, be = 0.0;
    unsigned sub_nz = 0u;
    // the shot numbers and blocks of 32 shots at a time: lane i loads those
    // of shot c0 + i (one coalesced load and one gather for 32 shots instead
    // of two dependent loads per shot), the loop takes them by shuffle
    for (uint64_t c0 = k0; c0 < k1; c0 += 32) {
        const uint64_t kl = c0 + (uint64_t)lane;
        const uint32_t s_l = kl < k1 ? order[kl] : 0u;
        const uint32_t b_l = kl < k1 ? shot_blk[s_l] : 0u;
        const int cnt = (int)min((uint64_t)32, k1 - c0);
        for (int i = 0; i < cnt; ++i) {
            const uint32_t s = __shfl_sync(0xffffffffu, s_l, i);
            const uint32_t blk = __shfl_sync(0xffffffffu, b_l, i);
            if (blk != cur) {
                cur = blk;
                Pl = warp_incl_scan(((uint32_t)lane < g.nsub) ? sub[(uint64_t)blk * g.nsub + lane] : 0.0, lane);
                be = bexcl[blk];
                const double prev = __shfl_up_sync(0xffffffffu, Pl, 1);
                const bool lane_nz = (uint32_t)lane < g.nsub && (lane == 0 ? Pl > 0.0 : Pl > prev);
                sub_nz = __ballot_sync(0xffffffffu, lane_nz);
            }
            const uint64_t base = (uint64_t)blk * bs;
            const double t = unif(seed, s) * tot;
            const unsigned hit = __ballot_sync(0xffffffffu, (uint32_t)lane < g.nsub && be + Pl > t);
            const uint32_t j = hit ? (uint32_t)(__ffs(hit) - 1) : (sub_nz ? (uint32_t)(31 - __clz(sub_nz)) : 0u);
            const double pj = __shfl_sync(0xffffffffu, Pl, (int)(j > 0 ? j - 1 : 0));
            const double pre = be + (j > 0 ? pj : 0.0);
            int first = -1, last_nz = -1;
            if (sizeof(R) == 4 && g.apl == 8) {
                lane_locate32(reinterpret_cast<const float *>(st), base, j, lane, pre, t, first, last_nz);
            } else {
                double p[8];
                lane_squares<R>(st, base, g, j, lane, p);
                double c[8], run = 0.0;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    run += p[e];
                    c[e] = run;
                }
                const double incl = warp_incl_scan(run, lane);
                const double start = pre + (incl - run);
#pragma unroll
                for (int e = 7; e >= 0; --e) {
                    if ((uint32_t)e < g.apl && start + c[e] > t) first = e;
                    if (last_nz < 0 && p[e] > 0.0) last_nz = e;
                }
            }
            const unsigned fl = __ballot_sync(0xffffffffu, first >= 0);
            uint64_t idx;
            if (fl) {
                const int L = __ffs(fl) - 1;
                idx = (uint64_t)L * g.apl + (uint64_t)__shfl_sync(0xffffffffu, first, L);
            } else {
                const unsigned nl = __ballot_sync(0xffffffffu, last_nz >= 0);
                const int L = nl ? 31 - __clz(nl) : 0;
                const int e = __shfl_sync(0xffffffffu, last_nz, L);
                idx = (uint64_t)L * g.apl + (uint64_t)(e > 0 ? e : 0);
            }
            if (lane == 0) out[s] = base + (uint64_t)j * g.sub + idx;
        }
    }
}

unsigned grid_for(uint64_t work, int threads, int num_sms)
{
    uint64_t g = (work + threads - 1) / threads;
    const uint64_t cap = (uint64_t)num_sms * 32;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// exclusive scan of nb values into out and their total into *total, on the
// handle's stream; cs holds 2 * ceil(nb / kScanChunk) values of scratch
template <typename T>
int scan_exclusive(qsim_state *s, const T *in, T *out, uint64_t nb, T *total, T *cs, const char *what)
{
    const uint64_t nc = (nb + kScanChunk - 1) / kScanChunk;
    launch_begin(s, KC_SAMPLE);
    k_scan_chunk_sums<T><<<(unsigned)nc, 256, 0, s->stream>>>(in, nb, cs);
    if (int rc = launch_end(s, what)) return rc;
    launch_begin(s, KC_SAMPLE);
    k_scan_exclusive<T><<<1, kScanThreads, 0, s->stream>>>(cs, cs + nc, nc, total);
    if (int rc = launch_end(s, what)) return rc;
    launch_begin(s, KC_SAMPLE);
    k_scan_chunk_out<T><<<(unsigned)nc, 256, 0, s->stream>>>(in, nb, cs + nc, out);
    return launch_end(s, what);
}

}  // namespace

uint64_t splitmix64_host(uint64_t x) { return smix(x); }
double uniform_host(uint64_t seed, uint64_t s) { return unif(seed, s); }

int launch_init_basis(qsim_state *s, uint64_t j)
{
    const size_t amp = (s->dtype == SIM_C128) ? 16 : 8;
    const uint64_t nvec = (uint64_t)(s->bytes / 16);
    uint64_t jvec;
    uint4 jval = make_uint4(0, 0, 0, 0);
    if (amp == 16) {
        jvec = j;
        const double one = 1.0;
        uint64_t bits;
        memcpy(&bits, &one, 8);
        jval.x = (uint32_t)bits; jval.y = (uint32_t)(bits >> 32);
    } else {
        jvec = j / 2;
        const float one = 1.0f;
        uint32_t bits;
        memcpy(&bits, &one, 4);
        if (j & 1) jval.z = bits; else jval.x = bits;
    }
    launch_begin(s, KC_INIT, (double)s->bytes);
    k_init_basis<<<grid_for(nvec, 256, s->num_sms), 256, 0, s->stream>>>((uint4 *)s->amps, nvec, jvec, jval);
    return launch_end(s, "init basis");
}

int reduce_sums(qsim_state *s, int mode, int qubit, double out[2])
{
    const uint64_t N = 1ull << s->n;
    const uint64_t nvec = (s->dtype == SIM_C128) ? N : N / 2;
    const uint64_t per = (nvec + kRedBlocks - 1) / kRedBlocks;
    launch_begin(s, KC_REDUCE, (double)s->bytes);
    if (s->dtype == SIM_C128) {
        const double *st = (const double *)s->amps;
        if (mode == RED_NORM) k_masked_sum<double, RED_NORM><<<kRedBlocks, kRedThreads, 0, s->stream>>>(st, nvec, per, qubit, s->n, s->red_partial);
        else if (mode == RED_BIT) k_masked_sum<double, RED_BIT><<<kRedBlocks, kRedThreads, 0, s->stream>>>(st, nvec, per, qubit, s->n, s->red_partial);
        else if (s->n >= 4) k_expz_chunks<double><<<kRedBlocks, kRedThreads, 0, s->stream>>>(st, N / 16, (N / 16 + kRedBlocks - 1) / kRedBlocks, s->n, s->red_partial);
        else k_masked_sum<double, RED_EXPZ><<<kRedBlocks, kRedThreads, 0, s->stream>>>(st, nvec, per, qubit, s->n, s->red_partial);
    } else {
        const float *st = (const float *)s->amps;
        if (mode == RED_NORM) k_sum_sq32<RED_NORM><<<kRedBlocks, kRedThreads, 0, s->stream>>>(st, nvec, per, qubit, s->red_partial);
        else if (mode == RED_BIT) k_sum_sq32<RED_BIT><<<kRedBlocks, kRedThreads, 0, s->stream>>>(st, nvec, per, qubit, s->red_partial);
        else if (s->n >= 4) k_expz32<<<kRedBlocks, kRedThreads, 0, s->stream>>>(st, N / 16, (N / 16 + kRedBlocks - 1) / kRedBlocks, s->n, s->red_partial);
        else k_masked_sum<float, RED_EXPZ><<<kRedBlocks, kRedThreads, 0, s->stream>>>(st, nvec, per, qubit, s->n, s->red_partial);
    }
    int rc = launch_end(s, "masked sum");
    if (rc) return rc;
    launch_begin(s, KC_REDUCE);
    k_final_sum<<<1, kRedThreads, 0, s->stream>>>(s->red_partial, kRedBlocks, s->red_out);
    rc = launch_end(s, "final sum");
    if (rc) return rc;
    QSIM_CUDA(cudaMemcpyAsync(s->host_red, s->red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    QSIM_CUDA(cudaStreamSynchronize(s->stream));
    out[0] = s->host_red[0];
    out[1] = s->host_red[1];
    return SIM_OK;
}

// sum_j |a_j|^2 into s->red_out[0] on the device (accumulated as for
// sim_norm), for kernels that read it later in stream order; no host sync
int reduce_norm_device(qsim_state *s)
{
    const uint64_t N = 1ull << s->n;
    const uint64_t nvec = (s->dtype == SIM_C128) ? N : N / 2;
    const uint64_t per = (nvec + kRedBlocks - 1) / kRedBlocks;
    launch_begin(s, KC_REDUCE, (double)s->bytes);
    if (s->dtype == SIM_C128)
        k_masked_sum<double, RED_NORM><<<kRedBlocks, kRedThreads, 0, s->stream>>>((const double *)s->amps, nvec, per, 0,
                                                                                  s->n, s->red_partial);
    else
        k_sum_sq32<RED_NORM><<<kRedBlocks, kRedThreads, 0, s->stream>>>((const float *)s->amps, nvec, per, 0,
                                                                       s->red_partial);
    if (int rc = launch_end(s, "norm pass")) return rc;
    launch_begin(s, KC_REDUCE);
    k_final_sum<<<1, kRedThreads, 0, s->stream>>>(s->red_partial, kRedBlocks, s->red_out);
    return launch_end(s, "norm final sum");
}

int launch_probabilities(qsim_state *s, void *dev_out, int out_real)
{
    const uint64_t N = 1ull << s->n;
    const unsigned g = grid_for(N, 256, s->num_sms);
    launch_begin(s, KC_PROB, (double)s->bytes + (double)N * (out_real == SIM_F64 ? 8.0 : 4.0));
    if (s->dtype == SIM_C128) {
        if (out_real == SIM_F64) k_probabilities<double, double><<<g, 256, 0, s->stream>>>((const double *)s->amps, N, (double *)dev_out);
        else k_probabilities<double, float><<<g, 256, 0, s->stream>>>((const double *)s->amps, N, (float *)dev_out);
    } else {
        if (out_real == SIM_F64) k_probabilities<float, double><<<g, 256, 0, s->stream>>>((const float *)s->amps, N, (double *)dev_out);
        else k_probabilities<float, float><<<g, 256, 0, s->stream>>>((const float *)s->amps, N, (float *)dev_out);
    }
    return launch_end(s, "probabilities");
}

int launch_collapse(qsim_state *s, int qubit, int outcome, double scale)
{
    const uint64_t N = 1ull << s->n;
    const unsigned g = grid_for(N, 256, s->num_sms);
    launch_begin(s, KC_COLLAPSE, 1.5 * (double)s->bytes);
    if (s->dtype == SIM_C128)
        k_collapse<double><<<g, 256, 0, s->stream>>>((double *)s->amps, N, qubit, outcome, scale);
    else
        k_collapse<float><<<g, 256, 0, s->stream>>>((float *)s->amps, N, qubit, outcome, (float)scale);
    return launch_end(s, "collapse");
}

bool sample_observe_fused(const qsim_state *s)
{
    return s->dtype == SIM_C64 && s->n >= kSampleLog && SubGeo(1ull << kSampleLog).sub == 256;
}

int run_sample(qsim_state *s, uint64_t shots, uint64_t seed, uint64_t *out, int out_on_device, double *norm_out,
               double *expz_out)
{
    if (shots == 0) return SIM_OK;
    const bool obs = expz_out != nullptr;
    if (obs && !sample_observe_fused(s)) return fail(SIM_EINVAL, "sample with <sum Z>: complex64, n >= 13 only");
    if (shots > 0xFFFFFFFFull) return fail(SIM_EINVAL, "sim_sample: at most 2^32 - 1 shots per call");
    const uint64_t N = 1ull << s->n;
    const uint64_t bs = (s->n >= kSampleLog) ? (1ull << kSampleLog) : N;
    const uint64_t nb = N / bs;
    const SubGeo sg(bs);
    // scratch: sub-sums (nb * nsub doubles), bsum, bexcl (nb doubles), counts, offs, cursor (nb u32),
    //          total, last (8 B each), shot_blk, order (shots u32), out (shots u64 for host output),
    //          chunk totals and offsets of the two scans
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
    const size_t o_sub = take(nb * sg.nsub * 8);
    const size_t o_bsum = take(nb * 8), o_bexcl = take(nb * 8), o_tot = take(8), o_last = take(8);
    const size_t o_cnt = take(nb * 4), o_offs = take(nb * 4), o_cur = take(nb * 4), o_u32tot = take(8);
    const size_t o_sblk = take(shots * 4), o_order = take(shots * 4);
    const uint64_t nchunk = (nb + kScanChunk - 1) / kScanChunk;
    const size_t o_cs = take(2 * nchunk * 8), o_cs32 = take(2 * nchunk * 4);
    const size_t o_zpart = obs ? take(2 * nb * 8) : 0, o_zout = obs ? take(2 * 8) : 0;
    const size_t o_out = out_on_device ? 0 : take(shots * 8);
    char *scratch = nullptr;
    QSIM_CUDA(cudaMallocAsync((void **)&scratch, off, s->stream));
    double *sub = (double *)(scratch + o_sub);
    double *bsum = (double *)(scratch + o_bsum), *bexcl = (double *)(scratch + o_bexcl);
    double *tot = (double *)(scratch + o_tot);
    uint64_t *last = (uint64_t *)(scratch + o_last);
    uint32_t *cnt = (uint32_t *)(scratch + o_cnt), *offs = (uint32_t *)(scratch + o_offs);
    uint32_t *cur = (uint32_t *)(scratch + o_cur), *u32tot = (uint32_t *)(scratch + o_u32tot);
    uint32_t *sblk = (uint32_t *)(scratch + o_sblk), *order = (uint32_t *)(scratch + o_order);
    uint64_t *dout = out_on_device ? out : (uint64_t *)(scratch + o_out);
    double *cs = (double *)(scratch + o_cs);
    uint32_t *cs32 = (uint32_t *)(scratch + o_cs32);
    double *zpart = obs ? (double *)(scratch + o_zpart) : nullptr, *zout = obs ? (double *)(scratch + o_zout) : nullptr;
    int rc = SIM_OK;
    const bool c128 = s->dtype == SIM_C128;
    do {
        launch_begin(s, KC_SAMPLE, (double)s->bytes);
        if (c128) k_sub_sums<double><<<(unsigned)nb, 256, 0, s->stream>>>((const double *)s->amps, bs, sub, bsum);
        else if (obs)
            k_sub_sums<float, true><<<(unsigned)nb, 256, 0, s->stream>>>((const float *)s->amps, bs, sub, bsum, s->n,
                                                                       zpart);
        else k_sub_sums<float><<<(unsigned)nb, 256, 0, s->stream>>>((const float *)s->amps, bs, sub, bsum);
        if ((rc = launch_end(s, "sub-block sums"))) break;
        if (obs) {
            launch_begin(s, KC_REDUCE);
            k_final_sum<<<1, kRedThreads, 0, s->stream>>>(zpart, (int)nb, zout);
            if ((rc = launch_end(s, "<sum Z> total"))) break;
        }
        if ((rc = scan_exclusive<double>(s, bsum, bexcl, nb, tot, cs, "block scan"))) break;
        launch_begin(s, KC_SAMPLE);
        k_last_nonzero<<<1, 32, 0, s->stream>>>(bsum, nb, last);
        if ((rc = launch_end(s, "last nonzero"))) break;
        // the host needs the last non-zero block as a launch argument: read it
        // together with the total (one small copy; the state stays on device)
        double htot = 0.0, hz = 0.0;
        uint64_t hlast = 0;
        if (cudaMemcpyAsync(&htot, tot, 8, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
            cudaMemcpyAsync(&hlast, last, 8, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
            (obs && cudaMemcpyAsync(&hz, zout, 8, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess) ||
            cudaStreamSynchronize(s->stream) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "sample readback");
            break;
        }
        if (norm_out) *norm_out = htot;
        if (expz_out) *expz_out = hz;
        if (!(htot > 0.0)) { rc = fail(SIM_EINVAL, "sim_sample: the state has zero norm"); break; }
        if (cudaMemsetAsync(cnt, 0, nb * 4, s->stream) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "memset"); break; }
        launch_begin(s, KC_SAMPLE);
        k_locate<<<grid_for(shots, 256, s->num_sms), 256, 0, s->stream>>>(shots, seed, bexcl, bsum, nb, tot, sblk,
                                                                           cnt, hlast);
        if ((rc = launch_end(s, "locate shots"))) break;
        if ((rc = scan_exclusive<uint32_t>(s, cnt, offs, nb, u32tot, cs32, "bucket scan"))) break;
        if (cudaMemcpyAsync(cur, offs, nb * 4, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "cursor copy");
            break;
        }
        launch_begin(s, KC_SAMPLE);
        k_scatter<<<grid_for(shots, 256, s->num_sms), 256, 0, s->stream>>>(shots, sblk, cur, order);
        if ((rc = launch_end(s, "scatter shots"))) break;
        // per shot: one sub-block of amplitudes; warps as many as are resident
        launch_begin(s, KC_SAMPLE, (double)shots * sg.sub * (c128 ? 16.0 : 8.0));
        {
            const void *fn = c128 ? (const void *)k_resolve<double> : (const void *)k_resolve<float>;
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0) != cudaSuccess || per_sm < 1)
                per_sm = 1;
            const uint64_t warps = (uint64_t)s->num_sms * per_sm * 8;
            const uint64_t per = (shots + warps - 1) / warps;
            const unsigned grid = (unsigned)((shots + per * 8 - 1) / (per * 8));
            if (c128)
                k_resolve<double><<<grid, 256, 0, s->stream>>>((const double *)s->amps, bs, seed, bexcl, tot, sub, sblk,
                                                               order, shots, per, dout);
            else
                k_resolve<float><<<grid, 256, 0, s->stream>>>((const float *)s->amps, bs, seed, bexcl, tot, sub, sblk,
                                                              order, shots, per, dout);
        }
        if ((rc = launch_end(s, "resolve shots"))) break;
        if (!out_on_device) {
            if (cudaMemcpyAsync(out, dout, shots * 8, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "shots readback");
                break;
            }
        }
    } while (0);
    cudaFreeAsync(scratch, s->stream);
    if (rc == SIM_OK && !out_on_device) QSIM_CUDA(cudaStreamSynchronize(s->stream));
    return rc;
}

}  // namespace qsim
