// density.cu -- density matrices and noise channels.
//
// The paper lists density matrices among what a simulator can return (§1)
// but describes no method for them; here they are built from the same
// pieces as the state vector.  The density matrix rho of n qubits is held as
// a 2n-qubit register: element rho[r][c] is amplitude (r << n) | c, so the
// column index takes register qubits 0 .. n-1 and the row index qubits
// n .. 2n-1.  Then
//   - a gate G on qubit t (rho -> G rho G^dagger) is G on register qubit
//     t + n (controls c + n) followed by conj(G) on register qubit t
//     (controls c): two commuting gates of the 2n-qubit register, which
//     every plan (per-gate, register tiles, fused tensor-core blocks, the
//     learned plan) applies unchanged;
//   - a single-qubit channel rho -> sum_m K_m rho K_m^dagger on qubit t is a
//     4 x 4 matrix on register qubits (t + n, t):
//       S[2r + c][2r' + c'] = sum_m K_m[r][r'] conj(K_m[c][c']),
//     applied by k_superop, one pass over the register;
//   - p_j = Re rho[j][j] sits at register index j (2^n + 1): trace, <sum Z>,
//     measurement and sampling read the diagonal into a complex128 vector of
//     2^n amplitudes sqrt(max(p_j, 0)) and run the state-vector reductions
//     and the sampler on it (squares of those roots are p_j to within an FP64
//     rounding); the collapse after a measurement keeps the block whose row
//     and column bit q both equal the outcome and divides it by p(outcome).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace qsim {

namespace {

constexpr int kDmThreads = 256;

template <typename R>
struct Super {
    R re[16], im[16];          // S[l][l'] at 4 l + l', l = 2 (row bit) + (column bit)
};

template <typename R> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

// y = S x for one group of four amplitudes (x[l], l = 2 (row bit) + column bit)
template <typename R>
__device__ __forceinline__ void super_apply(const Super<R> &S, R xr[4], R xi[4])
{
    R yr[4], yi[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        R ar = 0, ai = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ar += S.re[4 * l + k] * xr[k] - S.im[4 * l + k] * xi[k];
            ai += S.re[4 * l + k] * xi[k] + S.im[4 * l + k] * xr[k];
        }
        yr[l] = ar;
        yi[l] = ai;
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        xr[l] = yr[l];
        xi[l] = yi[l];
    }
}

__device__ __forceinline__ uint64_t insert2(uint64_t w, int a, int b)
{
    // zero bits inserted at a < b
    w = ((w >> a) << (a + 1)) | (w & ((1ull << a) - 1ull));
    w = ((w >> b) << (b + 1)) | (w & ((1ull << b) - 1ull));
    return w;
}

// One work item = the four amplitudes base | {0, 2^a, 2^b, 2^a + 2^b}, a < b
// (a = column qubit t, b = row qubit t + n).  complex64 with a >= 1 carries
// two neighbouring groups per item (16-byte vectors over bit 0); U items in
// flight per thread.
template <typename R, int VEC, int U>
__global__ void __launch_bounds__(kDmThreads) k_superop(R *__restrict__ st, uint64_t items, int a, int b, Super<R> S)
{
    const uint64_t first = (uint64_t)blockIdx.x * (kDmThreads * U) + threadIdx.x;
    const uint64_t oa = 1ull << a, ob = 1ull << b;
    if constexpr (VEC == 2) {
        float4 v[U][4];
        uint64_t base[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t w = first + (uint64_t)u * kDmThreads;
            base[u] = ~0ull;
            if (w < items) {
                base[u] = insert2(w * 2, a, b);
                v[u][0] = *reinterpret_cast<const float4 *>(st + 2 * base[u]);
                v[u][1] = *reinterpret_cast<const float4 *>(st + 2 * (base[u] | oa));
                v[u][2] = *reinterpret_cast<const float4 *>(st + 2 * (base[u] | ob));
                v[u][3] = *reinterpret_cast<const float4 *>(st + 2 * (base[u] | oa | ob));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (base[u] == ~0ull) continue;
            float xr[4], xi[4], zr[4], zi[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                xr[l] = v[u][l].x; xi[l] = v[u][l].y;
                zr[l] = v[u][l].z; zi[l] = v[u][l].w;
            }
            super_apply<float>(S, xr, xi);
            super_apply<float>(S, zr, zi);
            const uint64_t off[4] = {0, oa, ob, oa | ob};
#pragma unroll
            for (int l = 0; l < 4; ++l)
                *reinterpret_cast<float4 *>(st + 2 * (base[u] | off[l])) = make_float4(xr[l], xi[l], zr[l], zi[l]);
        }
    } else {
        using T = typename V2<R>::T;
        T v[U][4];
        uint64_t base[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t w = first + (uint64_t)u * kDmThreads;
            base[u] = ~0ull;
            if (w < items) {
                base[u] = insert2(w, a, b);
                v[u][0] = *reinterpret_cast<const T *>(st + 2 * base[u]);
                v[u][1] = *reinterpret_cast<const T *>(st + 2 * (base[u] | oa));
                v[u][2] = *reinterpret_cast<const T *>(st + 2 * (base[u] | ob));
                v[u][3] = *reinterpret_cast<const T *>(st + 2 * (base[u] | oa | ob));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (base[u] == ~0ull) continue;
            R xr[4], xi[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                xr[l] = v[u][l].x;
                xi[l] = v[u][l].y;
            }
            super_apply<R>(S, xr, xi);
            const uint64_t off[4] = {0, oa, ob, oa | ob};
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                T o;
                o.x = xr[l];
                o.y = xi[l];
                *reinterpret_cast<T *>(st + 2 * (base[u] | off[l])) = o;
            }
        }
    }
}

// complex64, channel on qubit 0 (a = 0): the column pair is one 16-byte
// vector, so an item is two vectors (row bit b = 0 and 1)
template <int U>
__global__ void __launch_bounds__(kDmThreads) k_superop_inner(float *__restrict__ st, uint64_t items, int b,
                                                              Super<float> S)
{
    const uint64_t first = (uint64_t)blockIdx.x * (kDmThreads * U) + threadIdx.x;
    const uint64_t ob = 1ull << b;
    float4 v[U][2];
    uint64_t base[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint64_t w = first + (uint64_t)u * kDmThreads;
        base[u] = ~0ull;
        if (w < items) {
            base[u] = insert2(w, 0, b);
            v[u][0] = *reinterpret_cast<const float4 *>(st + 2 * base[u]);
            v[u][1] = *reinterpret_cast<const float4 *>(st + 2 * (base[u] | ob));
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (base[u] == ~0ull) continue;
        float xr[4] = {v[u][0].x, v[u][0].z, v[u][1].x, v[u][1].z};
        float xi[4] = {v[u][0].y, v[u][0].w, v[u][1].y, v[u][1].w};
        super_apply<float>(S, xr, xi);
        *reinterpret_cast<float4 *>(st + 2 * base[u]) = make_float4(xr[0], xi[0], xr[1], xi[1]);
        *reinterpret_cast<float4 *>(st + 2 * (base[u] | ob)) = make_float4(xr[2], xi[2], xr[3], xi[3]);
    }
}

// root[j] = (sqrt(max(Re rho[j][j], 0)), 0) for j < 2^n
template <typename R>
__global__ void k_dm_diag_root(const R *__restrict__ rho, int n, uint64_t dim, double2 *__restrict__ root)
{
    const uint64_t stride = dim + 1;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < dim; j += (uint64_t)gridDim.x * blockDim.x) {
        const double p = (double)rho[2 * j * stride];
        root[j] = make_double2(sqrt(fmax(p, 0.0)), 0.0);
    }
}

// p[j] = Re rho[j][j]
template <typename R, typename O>
__global__ void k_dm_diag(const R *__restrict__ rho, uint64_t dim, O *__restrict__ p)
{
    const uint64_t stride = dim + 1;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < dim; j += (uint64_t)gridDim.x * blockDim.x)
        p[j] = (O)rho[2 * j * stride];
}

// keep rho[r][c] where bit q of r and of c equal m (scaled), zero the rest;
// one 16-byte vector per step (two complex64 or one complex128 amplitude)
template <typename R>
__global__ void k_dm_collapse(R *__restrict__ st, uint64_t nvec, int q, int n, int m, R scale)
{
    constexpr int AMPS = sizeof(R) == 4 ? 2 : 1;
    using T = typename V2<R>::T;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += (uint64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int e = 0; e < AMPS; ++e) {
            const uint64_t i = v * AMPS + e;
            const bool keep = (int)((i >> (q + n)) & 1) == m && (int)((i >> q) & 1) == m;
            T *p = reinterpret_cast<T *>(st) + i;
            if (keep) {
                T x = *p;
                x.x *= scale;
                x.y *= scale;
                *p = x;
            } else {
                T z;
                z.x = 0;
                z.y = 0;
                *p = z;
            }
        }
    }
}

// rho[r][c] = psi_r conj(psi_c)
template <typename R>
__global__ void k_dm_outer(const R *__restrict__ psi, int n, uint64_t total, R *__restrict__ rho)
{
    using T = typename V2<R>::T;
    const T *ps = reinterpret_cast<const T *>(psi);
    T *out = reinterpret_cast<T *>(rho);
    const uint64_t cm = (1ull << n) - 1ull;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const T a = ps[i >> n], b = ps[i & cm];
        T o;
        o.x = a.x * b.x + a.y * b.y;
        o.y = a.y * b.x - a.x * b.y;
        out[i] = o;
    }
}

unsigned dm_grid(uint64_t work, int num_sms)
{
    uint64_t g = (work + kDmThreads - 1) / kDmThreads;
    const uint64_t cap = (uint64_t)num_sms * 32;
    return (unsigned)std::max<uint64_t>(1, std::min(g, cap));
}

// 8 doubles per 2x2 matrix: (re, im) of [0][0], [0][1], [1][0], [1][1]
void superop_from_kraus(const double *kraus, int n_kraus, double S[32])
{
    for (int k = 0; k < 32; ++k) S[k] = 0.0;
    for (int m = 0; m < n_kraus; ++m) {
        const double *K = kraus + 8 * m;
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c)
                for (int r2 = 0; r2 < 2; ++r2)
                    for (int c2 = 0; c2 < 2; ++c2) {
                        const double ar = K[2 * (2 * r + r2)], ai = K[2 * (2 * r + r2) + 1];
                        const double br = K[2 * (2 * c + c2)], bi = -K[2 * (2 * c + c2) + 1];
                        const int idx = 4 * (2 * r + c) + (2 * r2 + c2);
                        S[2 * idx] += ar * br - ai * bi;
                        S[2 * idx + 1] += ar * bi + ai * br;
                    }
    }
}

}  // namespace

// the Kraus operators of a named channel (Nielsen & Chuang §8.3); returns the
// count (0 for an unknown kind)
int channel_kraus(int kind, double p, double out[32])
{
    for (int k = 0; k < 32; ++k) out[k] = 0.0;
    const double s = std::sqrt(1.0 - p), r = std::sqrt(p);
    switch (kind) {
    case SIM_CHANNEL_DEPOLARIZING: {
        const double a = std::sqrt(1.0 - 0.75 * p), q = std::sqrt(p / 4.0);
        out[0] = a; out[6] = a;                        // sqrt(1 - 3p/4) I
        out[8 + 2] = q; out[8 + 4] = q;                // sqrt(p/4) X
        out[16 + 3] = -q; out[16 + 5] = q;             // sqrt(p/4) Y
        out[24 + 0] = q; out[24 + 6] = -q;             // sqrt(p/4) Z
        return 4;
    }
    case SIM_CHANNEL_AMPLITUDE_DAMPING:
        out[0] = 1; out[6] = s;                        // diag(1, sqrt(1 - g))
        out[8 + 2] = r;                                // sqrt(g) |0><1|
        return 2;
    case SIM_CHANNEL_PHASE_DAMPING:
        out[0] = 1; out[6] = s;                        // diag(1, sqrt(1 - l))
        out[8 + 6] = r;                                // sqrt(l) |1><1|
        return 2;
    case SIM_CHANNEL_BIT_FLIP:
        out[0] = s; out[6] = s;
        out[8 + 2] = r; out[8 + 4] = r;
        return 2;
    case SIM_CHANNEL_PHASE_FLIP:
        out[0] = s; out[6] = s;
        out[8 + 0] = r; out[8 + 6] = -r;
        return 2;
    default:
        return 0;
    }
}

int launch_superop(qsim_state *s, int t, const double *kraus, int n_kraus)
{
    double S[32];
    superop_from_kraus(kraus, n_kraus, S);
    const int a = t, b = t + s->n_sys;
    const uint64_t groups = 1ull << (s->n - 2);
    const double amp = s->dtype == SIM_C128 ? 16.0 : 8.0;
    launch_begin(s, KC_CHANNEL, 2.0 * amp * 4.0 * (double)groups, 32.0 * 4.0 * (double)groups);
    if (s->dtype == SIM_C128) {
        Super<double> c;
        for (int k = 0; k < 16; ++k) { c.re[k] = S[2 * k]; c.im[k] = S[2 * k + 1]; }
        constexpr int U = 2;
        const uint64_t per = (uint64_t)kDmThreads * U;
        k_superop<double, 1, U><<<(unsigned)((groups + per - 1) / per), kDmThreads, 0, s->stream>>>(
            (double *)s->amps, groups, a, b, c);
    } else {
        Super<float> c;
        for (int k = 0; k < 16; ++k) { c.re[k] = (float)S[2 * k]; c.im[k] = (float)S[2 * k + 1]; }
        constexpr int U = 2;
        const uint64_t per = (uint64_t)kDmThreads * U;
        if (a >= 1) {
            const uint64_t items = groups / 2;
            k_superop<float, 2, U><<<(unsigned)((items + per - 1) / per), kDmThreads, 0, s->stream>>>(
                (float *)s->amps, items, a, b, c);
        } else {
            k_superop_inner<U><<<(unsigned)((groups + per - 1) / per), kDmThreads, 0, s->stream>>>(
                (float *)s->amps, groups, b, c);
        }
    }
    return launch_end(s, "channel");
}

namespace {

// a complex128 view of the diagonal roots, sharing s's stream and reduction
// scratch; the caller frees view->amps
int diag_view(qsim_state *s, qsim_state *v)
{
    const uint64_t dim = 1ull << s->n_sys;
    v->n = s->n_sys;
    v->dtype = SIM_C128;
    v->bytes = (size_t)16 * dim;
    v->stream = s->stream;
    v->device = s->device;
    v->num_sms = s->num_sms;
    v->red_partial = s->red_partial;
    v->red_out = s->red_out;
    v->host_red = s->host_red;
    v->dev_status = s->dev_status;
    v->profiling = false;
    QSIM_CUDA(cudaMallocAsync(&v->amps, v->bytes, s->stream));
    launch_begin(s, KC_PROB, (double)dim * (s->dtype == SIM_C128 ? 16.0 : 8.0) + (double)v->bytes);
    if (s->dtype == SIM_C128)
        k_dm_diag_root<double><<<dm_grid(dim, s->num_sms), kDmThreads, 0, s->stream>>>((const double *)s->amps,
                                                                                      s->n_sys, dim,
                                                                                      (double2 *)v->amps);
    else
        k_dm_diag_root<float><<<dm_grid(dim, s->num_sms), kDmThreads, 0, s->stream>>>((const float *)s->amps,
                                                                                     s->n_sys, dim,
                                                                                     (double2 *)v->amps);
    const int rc = launch_end(s, "density diagonal");
    if (rc) {
        cudaFreeAsync(v->amps, s->stream);
        v->amps = nullptr;
    }
    return rc;
}

void release_view(qsim_state *s, qsim_state *v)
{
    s->launches += v->launches;
    if (v->amps) cudaFreeAsync(v->amps, s->stream);
    v->amps = nullptr;
}

int check_dm(sim_t s, const char *who)
{
    if (!s) return fail(SIM_EINVAL, std::string(who) + ": null handle");
    if (!s->density) return fail(SIM_EINVAL, std::string(who) + ": not a density-matrix handle (sim_dm_create)");
    return SIM_OK;
}

bool is_channel_kind(int k) { return k >= SIM_GATE_CH_DEPOLARIZING && k <= SIM_GATE_CH_PHASE_FLIP; }

}  // namespace

}  // namespace qsim

using namespace qsim;

extern "C" {

int sim_dm_create(int n, int dtype, void *stream, sim_t *out)
{
    set_error("");
    if (!out) return fail(SIM_EINVAL, "sim_dm_create: out is NULL");
    *out = nullptr;
    if (n < 1 || n > 17) return fail(SIM_EINVAL, "sim_dm_create: n must be in [1, 17] (a 2n-qubit register)");
    sim_t s = nullptr;
    if (int rc = sim_create(2 * n, dtype, stream, &s)) return rc;
    s->density = true;
    s->n_sys = n;
    *out = s;
    return SIM_OK;
}

int sim_dm_create_from_buffer(int n, int dtype, void *dev_ptr, size_t bytes, void *stream, sim_t *out)
{
    set_error("");
    if (!out) return fail(SIM_EINVAL, "sim_dm_create_from_buffer: out is NULL");
    *out = nullptr;
    if (n < 1 || n > 17) return fail(SIM_EINVAL, "sim_dm_create_from_buffer: n must be in [1, 17]");
    sim_t s = nullptr;
    if (int rc = sim_create_from_buffer(2 * n, dtype, dev_ptr, bytes, stream, &s)) return rc;
    s->density = true;
    s->n_sys = n;
    *out = s;
    return SIM_OK;
}

int sim_dm_info(sim_t s, int *n)
{
    if (int rc = check_dm(s, "sim_dm_info")) return rc;
    if (n) *n = s->n_sys;
    return SIM_OK;
}

int sim_dm_set_basis_state(sim_t s, uint64_t j)
{
    if (int rc = check_dm(s, "sim_dm_set_basis_state")) return rc;
    if (j >> s->n_sys) return fail(SIM_EINVAL, "sim_dm_set_basis_state: j >= 2^n");
    return launch_init_basis(s, (j << s->n_sys) | j);
}

int sim_dm_set_pure(sim_t s, sim_t psi)
{
    if (int rc = check_dm(s, "sim_dm_set_pure")) return rc;
    if (!psi || psi->density) return fail(SIM_EINVAL, "sim_dm_set_pure: psi must be a state-vector handle");
    if (psi->n != s->n_sys || psi->dtype != s->dtype)
        return fail(SIM_EINVAL, "sim_dm_set_pure: psi must have n qubits and the same dtype");
    // psi's writes must land before this stream reads it
    if (psi->stream != s->stream) {
        cudaEvent_t e;
        QSIM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaEventRecord(e, psi->stream);
        cudaStreamWaitEvent(s->stream, e, 0);
        cudaEventDestroy(e);
    }
    const uint64_t total = 1ull << s->n;
    launch_begin(s, KC_INIT, (double)s->bytes);
    if (s->dtype == SIM_C128)
        k_dm_outer<double><<<dm_grid(total, s->num_sms), kDmThreads, 0, s->stream>>>((const double *)psi->amps,
                                                                                    s->n_sys, total, (double *)s->amps);
    else
        k_dm_outer<float><<<dm_grid(total, s->num_sms), kDmThreads, 0, s->stream>>>((const float *)psi->amps,
                                                                                   s->n_sys, total, (float *)s->amps);
    return launch_end(s, "density from pure state");
}

int sim_channel_kraus(int kind, double p, double *kraus, int *n_kraus)
{
    set_error("");
    if (!kraus || !n_kraus) return fail(SIM_EINVAL, "sim_channel_kraus: NULL output");
    if (!(p >= 0.0 && p <= 1.0)) return fail(SIM_EINVAL, "sim_channel_kraus: p must be in [0, 1]");
    double k[32];
    const int m = channel_kraus(kind, p, k);
    if (m == 0) return fail(SIM_EINVAL, "sim_channel_kraus: unknown channel kind");
    memcpy(kraus, k, sizeof(double) * 8 * m);
    *n_kraus = m;
    return SIM_OK;
}

int sim_dm_apply_kraus(sim_t s, int target, const double *kraus, int n_kraus)
{
    if (int rc = check_dm(s, "sim_dm_apply_kraus")) return rc;
    if (target < 0 || target >= s->n_sys) return fail(SIM_EINVAL, "sim_dm_apply_kraus: target out of range");
    if (!kraus || n_kraus < 1 || n_kraus > 16) return fail(SIM_EINVAL, "sim_dm_apply_kraus: 1..16 Kraus operators");
    for (int k = 0; k < 8 * n_kraus; ++k)
        if (!std::isfinite(kraus[k])) return fail(SIM_EINVAL, "sim_dm_apply_kraus: non-finite entry");
    return launch_superop(s, target, kraus, n_kraus);
}

int sim_dm_apply_channel(sim_t s, int kind, double p, int target)
{
    if (int rc = check_dm(s, "sim_dm_apply_channel")) return rc;
    if (target < 0 || target >= s->n_sys) return fail(SIM_EINVAL, "sim_dm_apply_channel: target out of range");
    if (!(p >= 0.0 && p <= 1.0)) return fail(SIM_EINVAL, "sim_dm_apply_channel: p must be in [0, 1]");
    double k[32];
    const int m = channel_kraus(kind, p, k);
    if (m == 0) return fail(SIM_EINVAL, "sim_dm_apply_channel: unknown channel kind");
    return launch_superop(s, target, k, m);
}

int sim_dm_apply_circuit(sim_t s, const sim_gate *gates, size_t n_gates, const sim_plan_opts *opts)
{
    if (int rc = check_dm(s, "sim_dm_apply_circuit")) return rc;
    if (n_gates == 0) return SIM_OK;
    if (!gates) return fail(SIM_EINVAL, "sim_dm_apply_circuit: gates is NULL");
    const int n = s->n_sys;
    for (size_t k = 0; k < n_gates; ++k) {
        const sim_gate &g = gates[k];
        char buf[80];
        snprintf(buf, sizeof buf, "sim_dm_apply_circuit: gate %zu: ", k);
        if (is_channel_kind(g.kind)) {
            if (g.target < 0 || g.target >= n) return fail(SIM_EINVAL, std::string(buf) + "target qubit out of range");
            if (g.n_controls != 0) return fail(SIM_EINVAL, std::string(buf) + "a channel takes no controls");
            if (!(g.params[0] >= 0.0 && g.params[0] <= 1.0))
                return fail(SIM_EINVAL, std::string(buf) + "channel parameter must be in [0, 1]");
            continue;
        }
        std::string why;
        if (validate_gate(n, g, &why)) return fail(SIM_EINVAL, buf + why);
    }
    sim_plan_opts o{};
    o.plan = SIM_PLAN_PER_GATE;
    if (opts) o = *opts;
    // each gate G on qubit t becomes G on the row qubit t + n and conj(G) on
    // the column qubit t
    auto lower_pair = [&](const sim_gate &g, sim_gate out[2]) {
        sim_gate row = g;
        row.target = g.target + n;
        if (g.kind == SIM_GATE_SWAP) row.target2 = g.target2 + n;
        for (int c = 0; c < g.n_controls; ++c) row.controls[c] = g.controls[c] + n;
        sim_gate col = g;
        if (g.kind != SIM_GATE_SWAP) {
            double m[8];
            gate_matrix(g.kind, g.params, g.matrix, m);
            col.kind = SIM_GATE_U;
            for (int e = 0; e < 8; ++e) col.matrix[e] = (e & 1) ? -m[e] : m[e];
        }
        out[0] = row;
        out[1] = col;
    };
    // which fused block size absorbs the channels (0: none).  The fused plan
    // does; the learned plan does when its model picks one fused variant for
    // every window of the gates without their channels.
    int absorb_k = 0;
    if (o.plan == SIM_PLAN_FUSED) {
        absorb_k = o.fuse_k ? o.fuse_k : (s->dtype == SIM_C128 ? 4 : 5);
    } else if (o.plan == SIM_PLAN_LEARNED && s->dtype == SIM_C128 && s->cost_model && s->n >= 11) {
        absorb_k = 4;
        s->last_plan.assign(1, 4);
    } else if (o.plan == SIM_PLAN_LEARNED && s->dtype == SIM_C64 && s->cost_model) {
        std::vector<sim_gate> reg;
        reg.reserve(2 * n_gates);
        for (size_t k = 0; k < n_gates; ++k) {
            if (is_channel_kind(gates[k].kind)) continue;
            sim_gate two[2];
            lower_pair(gates[k], two);
            reg.push_back(two[0]);
            reg.push_back(two[1]);
        }
        std::vector<int> best;
        if (!reg.empty()) {
            if (int rc = learned_choose(s, reg.data(), reg.size(), &best)) return rc;
            const int v = best.empty() ? -1 : best[0];
            bool same = v >= 3;
            for (int b : best) same = same && b == v;
            if (same) absorb_k = v;
        }
    }
    if (absorb_k) {
        // one pass per fused block, channels (4 x 4 on qubits t, t + n) inside
        // the blocks with the gates
        std::vector<SGate> lowered;
        std::vector<double> sup;
        for (size_t k = 0; k < n_gates; ++k) {
            const sim_gate &g = gates[k];
            if (is_channel_kind(g.kind)) {
                double kr[32], S[32];
                const int m = channel_kraus(g.kind - SIM_GATE_CH_DEPOLARIZING, g.params[0], kr);
                superop_from_kraus(kr, m, S);
                SGate x{OP_SUPER, g.target, 0ull, {}, (int)(sup.size() / 32)};
                x.target2 = g.target + n;
                sup.insert(sup.end(), S, S + 32);
                lowered.push_back(x);
                continue;
            }
            sim_gate two[2];
            lower_pair(g, two);
            lower_gates(two, 2, &lowered);
        }
        return apply_sgates_fused(s, lowered, sup.data(), absorb_k);
    }
    // runs of gates between channels under the plan; one pass per channel
    std::vector<sim_gate> reg;
    auto flush = [&]() -> int {
        if (reg.empty()) return SIM_OK;
        const int rc = apply_plan(s, reg.data(), reg.size(), o);
        reg.clear();
        return rc;
    };
    for (size_t k = 0; k < n_gates; ++k) {
        const sim_gate &g = gates[k];
        if (is_channel_kind(g.kind)) {
            if (int rc = flush()) return rc;
            double kr[32];
            const int m = channel_kraus(g.kind - SIM_GATE_CH_DEPOLARIZING, g.params[0], kr);
            if (int rc = launch_superop(s, g.target, kr, m)) return rc;
            continue;
        }
        sim_gate two[2];
        lower_pair(g, two);
        reg.push_back(two[0]);
        reg.push_back(two[1]);
    }
    return flush();
}

int sim_dm_probabilities(sim_t s, void *dev_out, int out_real)
{
    if (int rc = check_dm(s, "sim_dm_probabilities")) return rc;
    if (!dev_out) return fail(SIM_EINVAL, "sim_dm_probabilities: dev_out is NULL");
    if (out_real != SIM_F32 && out_real != SIM_F64) return fail(SIM_EINVAL, "sim_dm_probabilities: out_real");
    const uint64_t dim = 1ull << s->n_sys;
    const unsigned g = dm_grid(dim, s->num_sms);
    launch_begin(s, KC_PROB, (double)dim * ((s->dtype == SIM_C128 ? 16.0 : 8.0) + (out_real == SIM_F64 ? 8.0 : 4.0)));
    if (s->dtype == SIM_C128) {
        if (out_real == SIM_F64) k_dm_diag<double, double><<<g, kDmThreads, 0, s->stream>>>((const double *)s->amps, dim, (double *)dev_out);
        else k_dm_diag<double, float><<<g, kDmThreads, 0, s->stream>>>((const double *)s->amps, dim, (float *)dev_out);
    } else {
        if (out_real == SIM_F64) k_dm_diag<float, double><<<g, kDmThreads, 0, s->stream>>>((const float *)s->amps, dim, (double *)dev_out);
        else k_dm_diag<float, float><<<g, kDmThreads, 0, s->stream>>>((const float *)s->amps, dim, (float *)dev_out);
    }
    return launch_end(s, "density probabilities");
}

static int dm_diag_sum(sim_t s, int mode, int qubit, double out[2])
{
    qsim_state v;
    if (int rc = diag_view(s, &v)) return rc;
    const int rc = reduce_sums(&v, mode, qubit, out);
    release_view(s, &v);
    return rc;
}

int sim_dm_trace(sim_t s, double *out)
{
    if (int rc = check_dm(s, "sim_dm_trace")) return rc;
    if (!out) return fail(SIM_EINVAL, "sim_dm_trace: out is NULL");
    double r[2];
    if (int rc = dm_diag_sum(s, RED_NORM, 0, r)) return rc;
    *out = r[0];
    return SIM_OK;
}

int sim_dm_purity(sim_t s, double *out)
{
    if (int rc = check_dm(s, "sim_dm_purity")) return rc;
    if (!out) return fail(SIM_EINVAL, "sim_dm_purity: out is NULL");
    double r[2];
    if (int rc = reduce_sums(s, RED_NORM, 0, r)) return rc;
    *out = r[0];
    return SIM_OK;
}

int sim_dm_expect_z_sum(sim_t s, double *out)
{
    if (int rc = check_dm(s, "sim_dm_expect_z_sum")) return rc;
    if (!out) return fail(SIM_EINVAL, "sim_dm_expect_z_sum: out is NULL");
    double r[2];
    if (int rc = dm_diag_sum(s, RED_EXPZ, 0, r)) return rc;
    *out = r[0];
    return SIM_OK;
}

int sim_dm_measure(sim_t s, int qubit, uint64_t seed, uint64_t draw, int *outcome, double *prob)
{
    if (int rc = check_dm(s, "sim_dm_measure")) return rc;
    if (qubit < 0 || qubit >= s->n_sys) return fail(SIM_EINVAL, "sim_dm_measure: qubit out of range");
    double r[2];
    if (int rc = dm_diag_sum(s, RED_BIT, qubit, r)) return rc;
    const double p0 = r[0], p1 = r[1];
    if (!(p0 + p1 > 0.0)) return fail(SIM_EINVAL, "sim_dm_measure: the density matrix has zero trace");
    const double u = uniform_host(seed, draw);
    const int m = (p0 > u * (p0 + p1)) ? 0 : 1;
    const double pm = m ? p1 : p0;
    const uint64_t nvec = (uint64_t)(s->bytes / 16);
    launch_begin(s, KC_COLLAPSE, 1.25 * (double)s->bytes);
    if (s->dtype == SIM_C128)
        k_dm_collapse<double><<<dm_grid(nvec, s->num_sms), kDmThreads, 0, s->stream>>>((double *)s->amps, nvec, qubit,
                                                                                      s->n_sys, m, 1.0 / pm);
    else
        k_dm_collapse<float><<<dm_grid(nvec, s->num_sms), kDmThreads, 0, s->stream>>>((float *)s->amps, nvec, qubit,
                                                                                     s->n_sys, m, (float)(1.0 / pm));
    if (int rc = launch_end(s, "density collapse")) return rc;
    if (outcome) *outcome = m;
    if (prob) *prob = pm / (p0 + p1);
    return SIM_OK;
}

int sim_dm_sample(sim_t s, uint64_t shots, uint64_t seed, uint64_t *out, int out_on_device)
{
    if (int rc = check_dm(s, "sim_dm_sample")) return rc;
    if (shots > 0 && !out) return fail(SIM_EINVAL, "sim_dm_sample: out is NULL");
    if (shots == 0) return SIM_OK;
    qsim_state v;
    if (int rc = diag_view(s, &v)) return rc;
    int rc = run_sample(&v, shots, seed, out, out_on_device);
    release_view(s, &v);
    if (rc == SIM_OK && !out_on_device) QSIM_CUDA(cudaStreamSynchronize(s->stream));
    return rc;
}

}  // extern "C"
