// api.cu -- the C ABI: handles, validation, dispatch, measurement host logic,
// instrumentation.  Every entry point returns a sim_status and records a
// thread-local message on failure; nothing throws across the boundary.
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.cuh"

namespace qsim {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int status, const std::string &msg)
{
    set_error(msg);
    return status;
}

int cuda_fail(cudaError_t e, const char *what)
{
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    set_error(buf);
    return e == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA;
}

const char *kernel_class_name(int k)
{
    static const char *names[KC_COUNT] = {"init", "dense", "diag", "perm", "swap", "staged", "fused",
                                          "fuse_build", "prob", "reduce", "collapse", "sample", "batch", "mlp",
                                          "fused_multi", "fused_f16", "fused_c128", "channel"};
    return (k >= 0 && k < KC_COUNT) ? names[k] : "?";
}

static cudaEvent_t pool_event(qsim_state *s)
{
    if (s->event_next < s->event_pool.size()) return s->event_pool[s->event_next++];
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    s->event_pool.push_back(e);
    s->event_next = s->event_pool.size();
    return e;
}

void launch_begin(qsim_state *s, int cls, double alg_bytes, double alg_flops)
{
    if (!s->profiling) return;
    qsim_state::Mark m{cls, alg_bytes, alg_flops, pool_event(s), pool_event(s)};
    if (m.a) cudaEventRecord(m.a, s->stream);
    s->marks.push_back(m);
}

int launch_end(qsim_state *s, const char *what)
{
    s->launches++;
    if (s->profiling && !s->marks.empty() && s->marks.back().b) cudaEventRecord(s->marks.back().b, s->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    return SIM_OK;
}

int ensure_device(qsim_state *s, void **buf, size_t *cap, size_t need)
{
    if (*cap >= need) return SIM_OK;
    if (*buf) QSIM_CUDA(cudaFreeAsync(*buf, s->stream));
    *buf = nullptr;
    *cap = 0;
    size_t sz = need < 4096 ? 4096 : need;
    QSIM_CUDA(cudaMallocAsync(buf, sz, s->stream));
    *cap = sz;
    return SIM_OK;
}

int ensure_host_pinned(void **buf, size_t *cap, size_t need)
{
    if (*cap >= need) return SIM_OK;
    if (*buf) cudaFreeHost(*buf);
    *buf = nullptr;
    *cap = 0;
    size_t sz = need < 4096 ? 4096 : need;
    QSIM_CUDA(cudaMallocHost(buf, sz));
    *cap = sz;
    return SIM_OK;
}

static int amp_bytes(int dtype) { return dtype == SIM_C128 ? 16 : 8; }

// The L2 fetch granularity of this process's context on the device, set to
// 64 bytes once per device.  It is a hint that lives with the context (it
// does not outlast the process).  With the default, a load whose 64-byte run
// is the only used half of a 128-byte line (a gate whose lowest control or
// target is qubit 3) made the memory system fetch the whole line: measured at
// 30 qubits, CNOT and CZ with control 3 moved 1.5x their algorithmic bytes
// (0.70 of the copy peak) and reach 0.99 / 0.96 of it at 64 bytes; kernels
// that stream whole lines are unaffected.  A failure to set it is ignored.
static void set_l2_fetch_granularity(int device)
{
    static std::mutex m;
    static bool done[256] = {};
    std::lock_guard<std::mutex> lk(m);
    if (device < 0 || device >= 256 || done[device]) return;
    done[device] = true;
    if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, 64) != cudaSuccess) cudaGetLastError();
}

static int init_handle(qsim_state *s, void *stream)
{
    QSIM_CUDA(cudaGetDevice(&s->device));
    QSIM_CUDA(cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device));
    set_l2_fetch_granularity(s->device);
    if (stream) {
        s->stream = (cudaStream_t)stream;
        s->owns_stream = false;
    } else {
        QSIM_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
        s->owns_stream = true;
    }
    QSIM_CUDA(cudaMalloc((void **)&s->red_partial, sizeof(double) * 2 * kRedBlocks));
    QSIM_CUDA(cudaMalloc((void **)&s->red_out, sizeof(double) * 4));
    QSIM_CUDA(cudaMallocHost((void **)&s->host_red, sizeof(double) * 4));
    QSIM_CUDA(cudaMalloc((void **)&s->dev_status, sizeof(int) * 4));
    QSIM_CUDA(cudaMemset(s->dev_status, 0, sizeof(int) * 4));
    return SIM_OK;
}

static void free_handle(qsim_state *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->owns_amps && s->amps) cudaFree(s->amps);
    if (s->red_partial) cudaFree(s->red_partial);
    if (s->red_out) cudaFree(s->red_out);
    if (s->host_red) cudaFreeHost(s->host_red);
    if (s->dev_status) cudaFree(s->dev_status);
    if (s->dev_ops) cudaFree(s->dev_ops);
    if (s->host_ops) cudaFreeHost(s->host_ops);
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
    if (s->owns_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

static int check_handle(sim_t s)
{
    if (!s) return fail(SIM_EINVAL, "null handle");
    return SIM_OK;
}

// entry points whose meaning is that of a state vector
static int check_state(sim_t s, const char *who)
{
    if (!s) return fail(SIM_EINVAL, std::string(who) + ": null handle");
    if (s->density)
        return fail(SIM_EINVAL, std::string(who) + ": density-matrix handle (use the sim_dm_* entry points)");
    return SIM_OK;
}

int apply_plan(qsim_state *s, const sim_gate *gates, size_t n_gates, const sim_plan_opts &o)
{
    switch (o.plan) {
    case SIM_PLAN_PER_GATE:
        for (size_t k = 0; k < n_gates; ++k)
            if (int rc = launch_pair_gate(s, make_pair_gate(gates[k]))) return rc;
        return SIM_OK;
    case SIM_PLAN_STAGED:
        return apply_circuit_staged(s, gates, n_gates, o);
    case SIM_PLAN_FUSED:
        return apply_circuit_fused(s, gates, n_gates, o);
    case SIM_PLAN_LEARNED:
        return apply_circuit_learned(s, gates, n_gates, o);
    default:
        return fail(SIM_EINVAL, "sim_apply_circuit: unknown plan");
    }
}

}  // namespace qsim

using namespace qsim;

extern "C" {

const char *sim_last_error(void) { return g_last_error.c_str(); }
const char *sim_version(void) { return "qsim-gb300 0.1 (sm_103a)"; }
const char *sim_kernel_class_name(int k) { return kernel_class_name(k); }
int sim_num_kernel_classes(void) { return KC_COUNT; }

int sim_create(int n, int dtype, void *stream, sim_t *out)
{
    set_error("");
    if (!out) return fail(SIM_EINVAL, "sim_create: out is NULL");
    *out = nullptr;
    if (n < 1 || n > 34) return fail(SIM_EINVAL, "sim_create: n must be in [1, 34]");
    if (dtype != SIM_C64 && dtype != SIM_C128) return fail(SIM_EINVAL, "sim_create: unknown dtype");
    qsim_state *s = new (std::nothrow) qsim_state();
    if (!s) return fail(SIM_ENOMEM, "sim_create: host allocation");
    s->n = n;
    s->dtype = dtype;
    s->bytes = (size_t)amp_bytes(dtype) << n;
    int rc = init_handle(s, stream);
    if (rc) { free_handle(s); return rc; }
    size_t free_b = 0, total_b = 0;
    // QSIM_INJECT_ENOMEM (host-side fault injection for tests): behave as if
    // the device had no free memory, without touching the GPU allocator
    if (getenv("QSIM_INJECT_ENOMEM") != nullptr) {
        free_handle(s);
        return fail(SIM_ENOMEM, "sim_create: state does not fit in free device memory (injected)");
    }
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && s->bytes > free_b) {
        free_handle(s);
        return fail(SIM_ENOMEM, "sim_create: state does not fit in free device memory");
    }
    cudaError_t e = cudaMalloc(&s->amps, s->bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_handle(s);
        return fail(SIM_ENOMEM, "sim_create: device allocation of the state failed");
    }
    s->owns_amps = true;
    rc = launch_init_basis(s, 0);
    if (rc) { free_handle(s); return rc; }
    *out = s;
    return SIM_OK;
}

int sim_create_from_buffer(int n, int dtype, void *dev_ptr, size_t bytes, void *stream, sim_t *out)
{
    set_error("");
    if (!out) return fail(SIM_EINVAL, "sim_create_from_buffer: out is NULL");
    *out = nullptr;
    if (n < 1 || n > 34) return fail(SIM_EINVAL, "sim_create_from_buffer: n must be in [1, 34]");
    if (dtype != SIM_C64 && dtype != SIM_C128) return fail(SIM_EINVAL, "sim_create_from_buffer: unknown dtype");
    if (!dev_ptr || ((uintptr_t)dev_ptr & 15)) return fail(SIM_EINVAL, "sim_create_from_buffer: buffer must be 16-byte aligned");
    const size_t need = (size_t)amp_bytes(dtype) << n;
    if (bytes < need) return fail(SIM_EINVAL, "sim_create_from_buffer: buffer too small for 2^n amplitudes");
    qsim_state *s = new (std::nothrow) qsim_state();
    if (!s) return fail(SIM_ENOMEM, "host allocation");
    s->n = n;
    s->dtype = dtype;
    s->bytes = need;
    s->amps = dev_ptr;
    s->owns_amps = false;
    int rc = init_handle(s, stream);
    if (rc) { free_handle(s); return rc; }
    *out = s;
    return SIM_OK;
}

int sim_destroy(sim_t s)
{
    if (!s) return SIM_OK;
    free_handle(s);
    return SIM_OK;
}

int sim_state_info(sim_t s, int *n, int *dtype, void **dev_ptr, size_t *bytes)
{
    if (int rc = check_handle(s)) return rc;
    if (n) *n = s->n;
    if (dtype) *dtype = s->dtype;
    if (dev_ptr) *dev_ptr = s->amps;
    if (bytes) *bytes = s->bytes;
    return SIM_OK;
}

int sim_synchronize(sim_t s)
{
    if (int rc = check_handle(s)) return rc;
    QSIM_CUDA(cudaStreamSynchronize(s->stream));
    return SIM_OK;
}

int sim_set_basis_state(sim_t s, uint64_t j)
{
    if (int rc = check_state(s, "sim_set_basis_state")) return rc;
    if (j >> s->n) return fail(SIM_EINVAL, "sim_set_basis_state: j >= 2^n");
    return launch_init_basis(s, j);
}

int sim_load_state(sim_t s, const void *src, int src_is_host)
{
    if (int rc = check_handle(s)) return rc;
    if (!src) return fail(SIM_EINVAL, "sim_load_state: src is NULL");
    QSIM_CUDA(cudaMemcpyAsync(s->amps, src, s->bytes, src_is_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                              s->stream));
    if (src_is_host) QSIM_CUDA(cudaStreamSynchronize(s->stream));
    return SIM_OK;
}

int sim_copy_state(sim_t s, void *dst, int dst_is_host)
{
    if (int rc = check_handle(s)) return rc;
    if (!dst) return fail(SIM_EINVAL, "sim_copy_state: dst is NULL");
    QSIM_CUDA(cudaMemcpyAsync(dst, s->amps, s->bytes, dst_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                              s->stream));
    if (dst_is_host) QSIM_CUDA(cudaStreamSynchronize(s->stream));
    return SIM_OK;
}

int sim_apply_gate(sim_t s, const double U[8], int target, const int *controls, int n_controls)
{
    if (int rc = check_state(s, "sim_apply_gate")) return rc;
    if (!U) return fail(SIM_EINVAL, "sim_apply_gate: U is NULL");
    if (n_controls < 0 || n_controls > 2 || (n_controls > 0 && !controls))
        return fail(SIM_EINVAL, "sim_apply_gate: n_controls must be 0..2 with a controls array");
    sim_gate g;
    memset(&g, 0, sizeof g);
    g.kind = SIM_GATE_U;
    g.target = target;
    g.target2 = -1;
    g.n_controls = n_controls;
    g.controls[0] = n_controls > 0 ? controls[0] : -1;
    g.controls[1] = n_controls > 1 ? controls[1] : -1;
    memcpy(g.matrix, U, sizeof g.matrix);
    std::string why;
    if (validate_gate(s->n, g, &why)) return fail(SIM_EINVAL, "sim_apply_gate: " + why);
    return launch_pair_gate(s, make_pair_gate(g));
}

int sim_apply_circuit(sim_t s, const sim_gate *gates, size_t n_gates, const sim_plan_opts *opts)
{
    if (int rc = check_state(s, "sim_apply_circuit")) return rc;
    if (n_gates == 0) return SIM_OK;
    if (!gates) return fail(SIM_EINVAL, "sim_apply_circuit: gates is NULL");
    for (size_t k = 0; k < n_gates; ++k) {
        std::string why;
        if (validate_gate(s->n, gates[k], &why)) {
            char buf[64];
            snprintf(buf, sizeof buf, "sim_apply_circuit: gate %zu: ", k);
            return fail(SIM_EINVAL, buf + why);
        }
    }
    sim_plan_opts o{};
    o.plan = SIM_PLAN_PER_GATE;
    if (opts) o = *opts;
    return apply_plan(s, gates, n_gates, o);
}

int sim_probabilities(sim_t s, void *dev_out, int out_real)
{
    if (int rc = check_state(s, "sim_probabilities")) return rc;
    if (!dev_out) return fail(SIM_EINVAL, "sim_probabilities: dev_out is NULL");
    if (out_real != SIM_F32 && out_real != SIM_F64) return fail(SIM_EINVAL, "sim_probabilities: out_real");
    return launch_probabilities(s, dev_out, out_real);
}

int sim_norm(sim_t s, double *out)
{
    if (int rc = check_state(s, "sim_norm")) return rc;
    if (!out) return fail(SIM_EINVAL, "sim_norm: out is NULL");
    double r[2];
    if (int rc = reduce_sums(s, RED_NORM, 0, r)) return rc;
    *out = r[0];
    return SIM_OK;
}

int sim_expect_z_sum(sim_t s, double *out)
{
    if (int rc = check_state(s, "sim_expect_z_sum")) return rc;
    if (!out) return fail(SIM_EINVAL, "sim_expect_z_sum: out is NULL");
    double r[2];
    if (int rc = reduce_sums(s, RED_EXPZ, 0, r)) return rc;
    *out = r[0];
    return SIM_OK;
}

int sim_norm_expect_z(sim_t s, double *norm, double *expz)
{
    if (int rc = check_state(s, "sim_norm_expect_z")) return rc;
    if (!norm || !expz) return fail(SIM_EINVAL, "sim_norm_expect_z: NULL output");
    double r[2];
    if (int rc = reduce_sums(s, RED_EXPZ, 0, r)) return rc;
    *expz = r[0];
    *norm = r[1];
    return SIM_OK;
}

int sim_measure(sim_t s, int qubit, uint64_t seed, uint64_t draw, int *outcome, double *prob)
{
    if (int rc = check_state(s, "sim_measure")) return rc;
    if (qubit < 0 || qubit >= s->n) return fail(SIM_EINVAL, "sim_measure: qubit out of range");
    double r[2];
    if (int rc = reduce_sums(s, RED_BIT, qubit, r)) return rc;
    const double p0 = r[0], p1 = r[1];
    if (!(p0 + p1 > 0.0)) return fail(SIM_EINVAL, "sim_measure: the state has zero norm");
    const double u = uniform_host(seed, draw);
    const int m = (p0 > u * (p0 + p1)) ? 0 : 1;
    const double pm = m ? p1 : p0;
    if (int rc = launch_collapse(s, qubit, m, 1.0 / std::sqrt(pm))) return rc;
    if (outcome) *outcome = m;
    if (prob) *prob = pm / (p0 + p1);
    return SIM_OK;
}

int sim_sample(sim_t s, uint64_t shots, uint64_t seed, uint64_t *out, int out_on_device)
{
    if (int rc = check_state(s, "sim_sample")) return rc;
    if (shots > 0 && !out) return fail(SIM_EINVAL, "sim_sample: out is NULL");
    return run_sample(s, shots, seed, out, out_on_device);
}

int sim_sample_observe(sim_t s, uint64_t shots, uint64_t seed, uint64_t *out, int out_on_device, double *norm,
                       double *expz)
{
    if (int rc = check_state(s, "sim_sample_observe")) return rc;
    if (!norm || !expz) return fail(SIM_EINVAL, "sim_sample_observe: NULL norm or expz");
    if (shots > 0 && !out) return fail(SIM_EINVAL, "sim_sample_observe: out is NULL");
    // complex64 from 13 qubits: one pass gives the sub-block sums, the norm
    // (their total) and <sum Z>; otherwise the reduction pass runs first
    if (shots > 0 && sample_observe_fused(s)) return run_sample(s, shots, seed, out, out_on_device, norm, expz);
    double r[2];
    if (int rc = reduce_sums(s, RED_EXPZ, 0, r)) return rc;
    *expz = r[0];
    *norm = r[1];
    return run_sample(s, shots, seed, out, out_on_device);
}

int sim_plan_describe(int n, int dtype, const sim_gate *gates, size_t n_gates, const sim_plan_opts *opts,
                      int64_t *passes, int64_t *ops, int64_t *layout_changes, int32_t *order, size_t order_cap,
                      size_t *order_len)
{
    set_error("");
    if (n < 1 || n > 34) return fail(SIM_EINVAL, "sim_plan_describe: n must be in [1, 34]");
    if (n_gates && !gates) return fail(SIM_EINVAL, "sim_plan_describe: gates is NULL");
    for (size_t k = 0; k < n_gates; ++k) {
        std::string why;
        if (validate_gate(n, gates[k], &why)) return fail(SIM_EINVAL, "sim_plan_describe: " + why);
    }
    const int plan = opts ? opts->plan : SIM_PLAN_PER_GATE;
    if (plan == SIM_PLAN_FUSED) {
        // *passes: passes over the state; *ops: fused blocks
        if (layout_changes) *layout_changes = 0;
        if (order_len) *order_len = 0;
        int64_t blocks = 0, np = 0;
        const int rc = describe_fused(n, gates, n_gates, opts->fuse_k ? opts->fuse_k : (dtype == SIM_C128 ? 4 : 5), &blocks, 0,
                                      (opts->flags & SIM_FLAG_MULTI_BLOCK_PASSES) != 0, &np);
        if (passes) *passes = np;
        if (ops) *ops = blocks;
        return rc;
    }
    if (plan != SIM_PLAN_STAGED) return fail(SIM_EUNSUPPORTED, "sim_plan_describe: staged or fused plans only");
    return describe_staged(n, dtype, gates, n_gates, opts->tile_qubits, passes, ops, layout_changes, order,
                           order_cap, order_len);
}

int sim_plan_staged_ops(int n, int dtype, const sim_gate *gates, size_t n_gates, int tile_qubits, sim_tile_op *ops,
                        size_t ops_cap, int32_t *info, size_t info_cap, size_t *n_ops, size_t *n_passes)
{
    set_error("");
    if (n < 1 || n > 34) return fail(SIM_EINVAL, "sim_plan_staged_ops: n must be in [1, 34]");
    if (dtype != SIM_C64 && dtype != SIM_C128) return fail(SIM_EINVAL, "sim_plan_staged_ops: bad dtype");
    if (n_gates && !gates) return fail(SIM_EINVAL, "sim_plan_staged_ops: gates is NULL");
    for (size_t k = 0; k < n_gates; ++k) {
        std::string why;
        if (validate_gate(n, gates[k], &why)) return fail(SIM_EINVAL, "sim_plan_staged_ops: " + why);
    }
    return encode_staged(n, dtype, gates, n_gates, tile_qubits, ops, ops_cap, info, info_cap, n_ops, n_passes);
}

int sim_profile_enable(sim_t s, int on)
{
    if (int rc = check_handle(s)) return rc;
    s->profiling = on != 0;
    return SIM_OK;
}

int sim_profile_read(sim_t s, int max_classes, uint64_t *launches, double *total_ms, double *alg_bytes,
                     double *alg_flops, int reset)
{
    if (int rc = check_handle(s)) return rc;
    QSIM_CUDA(cudaStreamSynchronize(s->stream));
    for (const auto &m : s->marks) {
        float ms = 0.f;
        if (m.a && m.b && cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
            s->prof_launches[m.cls]++;
            s->prof_ms[m.cls] += ms;
            s->prof_bytes[m.cls] += m.bytes;
            s->prof_flops[m.cls] += m.flops;
        }
    }
    s->marks.clear();
    s->event_next = 0;
    for (int k = 0; k < max_classes && k < KC_COUNT; ++k) {
        if (launches) launches[k] = s->prof_launches[k];
        if (total_ms) total_ms[k] = s->prof_ms[k];
        if (alg_bytes) alg_bytes[k] = s->prof_bytes[k];
        if (alg_flops) alg_flops[k] = s->prof_flops[k];
    }
    if (reset) {
        for (int k = 0; k < KC_COUNT; ++k) { s->prof_launches[k] = 0; s->prof_ms[k] = 0; s->prof_bytes[k] = 0; s->prof_flops[k] = 0; }
    }
    return SIM_OK;
}

int sim_launch_count(sim_t s, uint64_t *out)
{
    if (int rc = check_handle(s)) return rc;
    if (out) *out = s->launches;
    return SIM_OK;
}

}  // extern "C"
