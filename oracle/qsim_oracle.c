/*
 * qsim_oracle.c -- plain, slow, FP64 CPU oracle for dense state-vector
 * gate application (Kelly, "Simulating Quantum Computers Using OpenCL",
 * arXiv:1805.00988).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg use it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Every routine is the plain definition of what the paper computes, written
 * for a reader to check by eye against the cited passage:
 *
 *   state layout      2^n complex amplitudes, amplitude j <-> basis |j>   (§2.1)
 *   qubit <-> bit     qubit t is bit t of the index (LSB = qubit 0); this is
 *                     how the App. B kernels and the App. C oracle loop
 *                     address qubits.
 *   gate              2x2 matrix [[A, B], [C, D]] row-major               (§2.2, App. B.1)
 *   application       Algorithm 1 (§2.3): for every index pair (a, b = a|2^t)
 *                     with bit t of a clear, update simultaneously
 *                     v_a <- A v_a + B v_b,  v_b <- C v_a + D v_b.
 *   controlled gate   §2.3: the update applies only where every control bit
 *                     is 1 (the paper has one control; two are allowed here).
 *   probabilities     App. B.3: p_j = |a_j|^2 (computed as re^2 + im^2).
 *   measurement       §1.3.3: p(m) = <psi|M_m^dag M_m|psi>, post-state
 *                     M_m psi / sqrt(p(m)), computational-basis projectors.
 *   sampling          §2.4: outcomes drawn from the probability vector, many
 *                     samples from one state, the state left unchanged.
 *
 * Readings where the paper is silent (gate conventions for U3/RX/RY/RZ/P,
 * the inverse-CDF selection rule, the SplitMix64 uniform draw) are stated at
 * each routine.
 *
 * Threading: the per-gate loop and the reductions carry an OpenMP pragma so
 * the same code can be timed on all host cores; the arithmetic per element is
 * identical with any thread count except for the reductions, which are always
 * serial (compensated) so results never depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Gate kinds known to the oracle.  The mapping from gate names is done by the
 * oracle's Python wrapper (oracle/__init__.py). */
enum {
    ORC_U = 0,     /* explicit 2x2 matrix given in mat[8] */
    ORC_X, ORC_Y, ORC_Z, ORC_H, ORC_S, ORC_SDG, ORC_T, ORC_TDG,
    ORC_RX, ORC_RY, ORC_RZ, ORC_P, ORC_U3,
    ORC_SWAP,
    ORC_NKINDS
};

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads the per-gate loops use from now on (t >= 1); for timing the same
 * code on one core and on all cores.  Results do not depend on it. */
void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t >= 1) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------------
 * Gate matrices, out[8] = (A.re, A.im, B.re, B.im, C.re, C.im, D.re, D.im).
 * H, X, Y, Z, S, T follow the gate table in §1.3.2.  The paper does not
 * define the rotations, so the standard conventions are read in:
 *   RX(t) = exp(-i t X / 2), RY(t) = exp(-i t Y / 2), RZ(t) = exp(-i t Z / 2),
 *   P(l)  = diag(1, e^{i l}) (the controlled form is the cu1 gate of App. A),
 *   U3(t, p, l) = [[cos t/2, -e^{i l} sin t/2], [e^{i p} sin t/2, e^{i(p+l)} cos t/2]].
 * Returns 0 on success, -1 for an unknown kind.
 * ---------------------------------------------------------------------- */
int orc_gate_matrix(int kind, const double *params, const double *mat, double *out)
{
    const double r2 = 1.0 / sqrt(2.0);
    double th = params ? params[0] : 0.0;
    double ph = params ? params[1] : 0.0;
    double la = params ? params[2] : 0.0;
    for (int k = 0; k < 8; ++k) out[k] = 0.0;
    switch (kind) {
    case ORC_U:
        for (int k = 0; k < 8; ++k) out[k] = mat[k];
        return 0;
    case ORC_X: out[2] = 1.0; out[4] = 1.0; return 0;
    case ORC_Y: out[3] = -1.0; out[5] = 1.0; return 0;            /* [[0,-i],[i,0]] */
    case ORC_Z: out[0] = 1.0; out[6] = -1.0; return 0;
    case ORC_H: out[0] = r2; out[2] = r2; out[4] = r2; out[6] = -r2; return 0;
    case ORC_S: out[0] = 1.0; out[7] = 1.0; return 0;             /* diag(1, i) */
    case ORC_SDG: out[0] = 1.0; out[7] = -1.0; return 0;          /* diag(1, -i) */
    case ORC_T: out[0] = 1.0; out[6] = cos(M_PI / 4); out[7] = sin(M_PI / 4); return 0;
    case ORC_TDG: out[0] = 1.0; out[6] = cos(M_PI / 4); out[7] = -sin(M_PI / 4); return 0;
    case ORC_RX:
        out[0] = cos(th / 2); out[3] = -sin(th / 2);
        out[5] = -sin(th / 2); out[6] = cos(th / 2);
        return 0;
    case ORC_RY:
        out[0] = cos(th / 2); out[2] = -sin(th / 2);
        out[4] = sin(th / 2); out[6] = cos(th / 2);
        return 0;
    case ORC_RZ:
        out[0] = cos(th / 2); out[1] = -sin(th / 2);
        out[6] = cos(th / 2); out[7] = sin(th / 2);
        return 0;
    case ORC_P:
        out[0] = 1.0; out[6] = cos(th); out[7] = sin(th);
        return 0;
    case ORC_U3: {
        double c = cos(th / 2), s = sin(th / 2);
        out[0] = c;
        out[2] = -cos(la) * s; out[3] = -sin(la) * s;
        out[4] = cos(ph) * s;  out[5] = sin(ph) * s;
        out[6] = cos(ph + la) * c; out[7] = sin(ph + la) * c;
        return 0;
    }
    default:
        return -1;
    }
}

/* all control bits of index i set? */
static int controls_set(uint64_t i, int nctrl, const int *ctrl)
{
    for (int c = 0; c < nctrl; ++c)
        if (!((i >> ctrl[c]) & 1u)) return 0;
    return 1;
}

/* ------------------------------------------------------------------------
 * Algorithm 1 (§2.3) with the controlled restriction of §2.3, applied in
 * place to psi (interleaved re, im; 2^n amplitudes).  Visits every index i of
 * the register; the pairs are those i whose bit t is 0 and whose control bits
 * are all 1, with partner j = i | 2^t.  Both rows use the old values.
 * ---------------------------------------------------------------------- */
static void apply_2x2(int n, double *psi, int t, int nctrl, const int *ctrl, const double *g)
{
    const uint64_t N = (uint64_t)1 << n;
    const uint64_t tb = (uint64_t)1 << t;
    const double Ar = g[0], Ai = g[1], Br = g[2], Bi = g[3];
    const double Cr = g[4], Ci = g[5], Dr = g[6], Di = g[7];
    int64_t iN = (int64_t)N;
#pragma omp parallel for schedule(static)
    for (int64_t ii = 0; ii < iN; ++ii) {
        uint64_t i = (uint64_t)ii;
        if (i & tb) continue;
        if (!controls_set(i, nctrl, ctrl)) continue;
        uint64_t j = i | tb;
        double ar = psi[2 * i], ai = psi[2 * i + 1];
        double br = psi[2 * j], bi = psi[2 * j + 1];
        /* v_a <- A v_a + B v_b */
        double nar = (Ar * ar - Ai * ai) + (Br * br - Bi * bi);
        double nai = (Ar * ai + Ai * ar) + (Br * bi + Bi * br);
        /* v_b <- C v_a + D v_b  (old v_a) */
        double nbr = (Cr * ar - Ci * ai) + (Dr * br - Di * bi);
        double nbi = (Cr * ai + Ci * ar) + (Dr * bi + Di * br);
        psi[2 * i] = nar; psi[2 * i + 1] = nai;
        psi[2 * j] = nbr; psi[2 * j + 1] = nbi;
    }
}

/* SWAP(a, b), optionally controlled: exchange the amplitudes of the index
 * pairs that differ only in bits a and b, with (bit a, bit b) = (1, 0) and
 * (0, 1).  This is the permutation matrix of the two-qubit SWAP; the paper
 * uses it nowhere, the QFT's closing qubit reversal does. */
static void apply_swap(int n, double *psi, int a, int b, int nctrl, const int *ctrl)
{
    const uint64_t N = (uint64_t)1 << n;
    const uint64_t ab = (uint64_t)1 << a, bb = (uint64_t)1 << b;
    int64_t iN = (int64_t)N;
#pragma omp parallel for schedule(static)
    for (int64_t ii = 0; ii < iN; ++ii) {
        uint64_t i = (uint64_t)ii;
        if (!(i & ab) || (i & bb)) continue;      /* i has bit a = 1, bit b = 0 */
        if (!controls_set(i, nctrl, ctrl)) continue;
        uint64_t j = (i & ~ab) | bb;              /* bit a = 0, bit b = 1 */
        double r = psi[2 * i], m = psi[2 * i + 1];
        psi[2 * i] = psi[2 * j]; psi[2 * i + 1] = psi[2 * j + 1];
        psi[2 * j] = r; psi[2 * j + 1] = m;
    }
}

/* Check the qubit arguments of one gate; returns 0 when valid. */
static int check_gate(int n, int kind, int t, int t2, int nctrl, const int *ctrl)
{
    if (kind < 0 || kind >= ORC_NKINDS) return -1;
    if (t < 0 || t >= n) return -1;
    if (nctrl < 0 || nctrl > 2) return -1;
    if (kind == ORC_SWAP && (t2 < 0 || t2 >= n || t2 == t)) return -1;
    for (int c = 0; c < nctrl; ++c) {
        if (ctrl[c] < 0 || ctrl[c] >= n || ctrl[c] == t) return -1;
        if (kind == ORC_SWAP && ctrl[c] == t2) return -1;
        for (int d = 0; d < c; ++d)
            if (ctrl[d] == ctrl[c]) return -1;
    }
    return 0;
}

/* Apply m gates in order.  ctrl is m x 2, params m x 3, mat m x 8.
 * Returns 0, or -(g+1) for the first invalid gate g (state untouched from
 * that gate on). */
int orc_apply_circuit(int n, double *psi, int64_t m, const int *kind, const int *target,
                      const int *target2, const int *nctrl, const int *ctrl,
                      const double *params, const double *mat)
{
    for (int64_t g = 0; g < m; ++g) {
        if (check_gate(n, kind[g], target[g], target2[g], nctrl[g], ctrl + 2 * g))
            return (int)(-(g + 1));
        if (kind[g] == ORC_SWAP) {
            apply_swap(n, psi, target[g], target2[g], nctrl[g], ctrl + 2 * g);
        } else {
            double u[8];
            orc_gate_matrix(kind[g], params + 3 * g, mat + 8 * g, u);
            apply_2x2(n, psi, target[g], nctrl[g], ctrl + 2 * g, u);
        }
    }
    return 0;
}

/* |0...0> or any basis state |j> (§2.1: a new register starts in |00...0>). */
void orc_basis_state(int n, double *psi, uint64_t j)
{
    const uint64_t N = (uint64_t)1 << n;
    memset(psi, 0, sizeof(double) * 2 * N);
    psi[2 * j] = 1.0;
}

/* App. B.3: p_j = |a_j|^2, here re^2 + im^2. */
void orc_probabilities(int n, const double *psi, double *p)
{
    const uint64_t N = (uint64_t)1 << n;
    for (uint64_t i = 0; i < N; ++i)
        p[i] = psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
}

/* Neumaier's compensated summation (Neumaier 1974), serial, so the result does
 * not depend on a thread count. */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nsum_get(const nsum *a) { return a->s + a->c; }

/* squared norm sum_j |a_j|^2 (the normalisation condition of §1.3.1). */
double orc_norm2(int n, const double *psi)
{
    const uint64_t N = (uint64_t)1 << n;
    nsum acc = {0, 0};
    for (uint64_t i = 0; i < N; ++i)
        nsum_add(&acc, psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1]);
    return nsum_get(&acc);
}

/* probability mass with bit q equal to 1 (p(1) of §1.3.3 for qubit q,
 * unnormalised). */
double orc_prob_one(int n, const double *psi, int q)
{
    const uint64_t N = (uint64_t)1 << n;
    nsum acc = {0, 0};
    for (uint64_t i = 0; i < N; ++i)
        if ((i >> q) & 1u)
            nsum_add(&acc, psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1]);
    return nsum_get(&acc);
}

/* ------------------------------------------------------------------------
 * SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): one step from state x adds the golden gamma
 * 0x9E3779B97F4A7C15 and applies the variant-13 mix.  Draw s of a stream with
 * seed S is u_s = (splitmix64(S + s) >> 11) * 2^-53, uniform in [0, 1).
 * ---------------------------------------------------------------------- */
uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double orc_uniform(uint64_t seed, uint64_t s)
{
    return (double)(orc_splitmix64(seed + s) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------
 * Single-qubit measurement in the computational basis (§1.3.3): p(0), p(1)
 * from the projectors |0><0|, |1><1| on qubit q.  The outcome is chosen by
 * inverse CDF over (0, 1): outcome 0 iff p0 > u * (p0 + p1), with
 * u = orc_uniform(seed, draw).  Post-state M_m psi / sqrt(p(m)): the other
 * half is zeroed and the kept half divided by sqrt of its mass, so the
 * result has unit norm.  Returns the outcome; *p_out gets p(m) / (p0 + p1).
 * ---------------------------------------------------------------------- */
int orc_measure(int n, double *psi, int q, uint64_t seed, uint64_t draw, double *p_out)
{
    const uint64_t N = (uint64_t)1 << n;
    double total = orc_norm2(n, psi);
    double p1 = orc_prob_one(n, psi, q);
    double p0 = total - p1;
    {
        /* p0 as its own compensated sum, so it does not inherit the
         * cancellation error of total - p1 */
        nsum acc = {0, 0};
        for (uint64_t i = 0; i < N; ++i)
            if (!((i >> q) & 1u))
                nsum_add(&acc, psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1]);
        p0 = nsum_get(&acc);
    }
    double u = orc_uniform(seed, draw);
    int outcome = (p0 > u * (p0 + p1)) ? 0 : 1;
    double pm = outcome ? p1 : p0;
    double scale = 1.0 / sqrt(pm);
    for (uint64_t i = 0; i < N; ++i) {
        if ((int)((i >> q) & 1u) == outcome) {
            psi[2 * i] *= scale; psi[2 * i + 1] *= scale;
        } else {
            psi[2 * i] = 0.0; psi[2 * i + 1] = 0.0;
        }
    }
    if (p_out) *p_out = pm / (p0 + p1);
    return outcome;
}

/* ------------------------------------------------------------------------
 * Shot sampling (§2.4): probabilities p_i (App. B.3), inclusive prefix
 * C_i = p_0 + ... + p_i accumulated serially with Neumaier compensation, and
 * for shot s the outcome is the smallest i with C_i > u_s * C_{N-1},
 * u_s = orc_uniform(seed, s).  If rounding leaves no such i, the last index
 * with p_i > 0 is taken.  The state is not changed.
 * ---------------------------------------------------------------------- */
int orc_sample(int n, const double *psi, uint64_t shots, uint64_t seed, uint64_t *out)
{
    const uint64_t N = (uint64_t)1 << n;
    double *C = (double *)malloc(sizeof(double) * N);
    if (!C) return -1;
    nsum acc = {0, 0};
    uint64_t last_nz = 0;
    for (uint64_t i = 0; i < N; ++i) {
        double p = psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
        if (p > 0) last_nz = i;
        nsum_add(&acc, p);
        C[i] = nsum_get(&acc);
    }
    double total = C[N - 1];
    for (uint64_t s = 0; s < shots; ++s) {
        double target = orc_uniform(seed, s) * total;
        /* smallest i with C[i] > target (C is non-decreasing) */
        uint64_t lo = 0, hi = N;            /* answer in [lo, hi] ; hi = none */
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (C[mid] > target) hi = mid; else lo = mid + 1;
        }
        out[s] = (lo < N) ? lo : last_nz;
    }
    free(C);
    return 0;
}

/* ------------------------------------------------------------------------
 * The same inverse-CDF rule on given weights p_0 .. p_{N-1} >= 0 (a density
 * matrix's diagonal, §1.3.3 with M_j = |j><j|): compensated inclusive prefix
 * C_i, shot s -> smallest i with C_i > u_s C_{N-1}, else the last i with
 * p_i > 0.
 * ---------------------------------------------------------------------- */
int orc_sample_weights(uint64_t N, const double *p, uint64_t shots, uint64_t seed, uint64_t *out)
{
    double *C = (double *)malloc(sizeof(double) * (N ? N : 1));
    if (!C) return -1;
    nsum acc = {0, 0};
    uint64_t last_nz = 0;
    for (uint64_t i = 0; i < N; ++i) {
        if (p[i] > 0) last_nz = i;
        nsum_add(&acc, p[i]);
        C[i] = nsum_get(&acc);
    }
    double total = N ? C[N - 1] : 0.0;
    for (uint64_t s = 0; s < shots; ++s) {
        double target = orc_uniform(seed, s) * total;
        uint64_t lo = 0, hi = N;
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (C[mid] > target) hi = mid; else lo = mid + 1;
        }
        out[s] = (lo < N) ? lo : last_nz;
    }
    free(C);
    return 0;
}

/* <sum_i Z_i> = sum_x p_x (n - 2 popcount(x)): Z_i has eigenvalue +1 on
 * bit i = 0 and -1 on bit i = 1 (the gate table of §1.3.2). */
double orc_expect_z_sum(int n, const double *psi)
{
    const uint64_t N = (uint64_t)1 << n;
    nsum acc = {0, 0};
    for (uint64_t x = 0; x < N; ++x) {
        double p = psi[2 * x] * psi[2 * x] + psi[2 * x + 1] * psi[2 * x + 1];
        int pc = 0;
        for (int b = 0; b < n; ++b) pc += (int)((x >> b) & 1u);
        nsum_add(&acc, p * (double)(n - 2 * pc));
    }
    return nsum_get(&acc);
}

/* infidelity 1 - |<a|b>|^2 / (<a|a><b|b>), FP64, compensated sums. */
double orc_infidelity(int n, const double *a, const double *b)
{
    const uint64_t N = (uint64_t)1 << n;
    nsum re = {0, 0}, im = {0, 0}, na = {0, 0}, nb = {0, 0};
    for (uint64_t i = 0; i < N; ++i) {
        double ar = a[2 * i], ai = a[2 * i + 1], br = b[2 * i], bi = b[2 * i + 1];
        /* conj(a) * b */
        nsum_add(&re, ar * br + ai * bi);
        nsum_add(&im, ar * bi - ai * br);
        nsum_add(&na, ar * ar + ai * ai);
        nsum_add(&nb, br * br + bi * bi);
    }
    double r = nsum_get(&re), m = nsum_get(&im);
    return 1.0 - (r * r + m * m) / (nsum_get(&na) * nsum_get(&nb));
}
