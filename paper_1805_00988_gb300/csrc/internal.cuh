// internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <atomic>
#include <thread>
#include <algorithm>
#include <memory>
#include <vector>

#include "../../include/qsim_gb300.h"

namespace qsim {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
int fail(int status, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define QSIM_CUDA(call)                                                   \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return ::qsim::cuda_fail(e_, #call);       \
    } while (0)

// ---------------------------------------------------------------- kernel classes
// Every launch is tagged with one class for launch counting and profiling.
enum KernelClass {
    KC_INIT = 0,
    KC_DENSE,        // dense 2x2 on amplitude pairs (Algorithm 1)
    KC_DIAG,         // diagonal / phase gates
    KC_PERM,         // X / CNOT / Toffoli moves and antidiagonal gates
    KC_SWAP,
    KC_STAGED,       // multi-gate tile pass
    KC_FUSED,        // fused k-qubit unitary apply
    KC_FUSE_BUILD,   // FP64 fused-unitary construction
    KC_PROB,         // probabilities
    KC_REDUCE,       // norm / masked sums / <Z> partial reductions
    KC_COLLAPSE,
    KC_SAMPLE,       // block sums, scans, shot location, resolution
    KC_BATCH,        // batched persistent circuits
    KC_MLP,          // cost-model forward / backward / Adam
    KC_FUSED_MULTI,  // several fused blocks applied per pass over the state
    KC_FUSED_F16,    // fused 6-qubit unitary apply on FP16-split operands
    KC_FUSED_C128,   // fused 4-qubit unitary apply to complex128 states on integer digit planes
    KC_CHANNEL,      // density matrices: single-qubit channel (4 x 4 superoperator) pass
    KC_COUNT
};
const char *kernel_class_name(int k);

}  // namespace qsim

// ---------------------------------------------------------------- handle
struct qsim_state {
    int n = 0;
    int dtype = SIM_C64;
    void *amps = nullptr;
    size_t bytes = 0;
    bool owns_amps = false;
    bool owns_stream = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    // FP64 reduction scratch (partials of fixed-grid reductions), owned
    double *red_partial = nullptr;   // kRedBlocks * 4 doubles
    double *red_out = nullptr;       // 4 doubles
    double *host_red = nullptr;      // pinned, 4 doubles
    int *dev_status = nullptr;       // device status word of bounded waits (0 = ok)
    bool density = false;            // a density matrix of n_sys qubits held as an n = 2 n_sys register
    int n_sys = 0;
    void *cost_model = nullptr;      // qsim_mlp used by SIM_PLAN_LEARNED (not owned)
    std::vector<int> last_plan;      // variant chosen per window by the last learned plan
    // circuit upload buffers (device), grown on demand
    void *dev_ops = nullptr;
    size_t dev_ops_bytes = 0;
    void *host_ops = nullptr;        // pinned staging
    size_t host_ops_bytes = 0;
    // instrumentation
    uint64_t launches = 0;
    bool profiling = false;
    struct Mark { int cls; double bytes, flops; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> event_pool;
    size_t event_next = 0;
    uint64_t prof_launches[qsim::KC_COUNT] = {0};
    double prof_ms[qsim::KC_COUNT] = {0};
    double prof_bytes[qsim::KC_COUNT] = {0};
    double prof_flops[qsim::KC_COUNT] = {0};
};

namespace qsim {

constexpr int kRedBlocks = 1216;     // 152 SMs x 8 blocks: fixed grid for deterministic FP64 sums
constexpr int kRedThreads = 256;

// Launch bracketing: call begin() before and end() after each kernel launch.
// alg_bytes = the bytes the launch must move at minimum (what the operation
// reads and writes of the state), used for roofline accounting.
void launch_begin(qsim_state *s, int cls, double alg_bytes = 0.0, double alg_flops = 0.0);
struct SGate;
// algorithmic floating-point operations of one lowered gate on an n-qubit state
// (8 per complex multiply-add; sign flips and moves count 0)
double sgate_flops(const SGate &g, int n);
int launch_end(qsim_state *s, const char *what);

// ---------------------------------------------------------------- per-gate kernels
// Classified gate, ready for a per-gate launch.
enum GateOp { OP_DENSE = 0, OP_DIAG, OP_DIAG_HI, OP_ANTIDIAG, OP_XPERM, OP_SWAP, OP_IDENTITY,
              OP_SUPER   // a 4 x 4 matrix on two qubits (a density matrix's channel), fused plans only
};

struct PairGate {
    int op;
    int target;            // qubit t (first qubit of a swap)
    int target2;           // swap partner
    int nctrl;
    int ctrl[2];
    double m[8];           // A, B, C, D (re, im)
};

// Classify a 2x2 matrix (exact comparisons): identity, diagonal, phase on |1>,
// pure X, antidiagonal or dense.
int classify_matrix(const double m[8]);

// Build the matrix of a named gate kind; returns 0 or -1 for an unknown kind.
int gate_matrix(int kind, const double *params, const double *matrix, double out[8]);

// Validate one ABI gate for an n-qubit register.
int validate_gate(int n, const sim_gate &g, std::string *why);

// Turn an ABI gate into a classified PairGate.
PairGate make_pair_gate(const sim_gate &g);

int launch_pair_gate(qsim_state *s, const PairGate &g);

// a validated gate list on the handle's register under plan o (the dispatch
// of sim_apply_circuit, without the handle-kind check)
int apply_plan(qsim_state *s, const sim_gate *gates, size_t n_gates, const sim_plan_opts &o);

// density matrices (density.cu): Kraus operators of a named channel
// (SIM_CHANNEL_*; returns their count, 0 for an unknown kind) and one channel
// pass on system qubit t of a density handle
int channel_kraus(int kind, double p, double out[32]);
int launch_superop(qsim_state *s, int t, const double *kraus, int n_kraus);

// ---------------------------------------------------------------- reductions
// mode for masked FP64 sums of |a|^2
enum RedMode { RED_NORM = 0, RED_BIT = 1, RED_EXPZ = 2 };
int launch_init_basis(qsim_state *s, uint64_t j);
int reduce_sums(qsim_state *s, int mode, int qubit, double out[2]);
// sum_j |a_j|^2 into s->red_out[0] on the device, no host sync (stream-ordered)
int reduce_norm_device(qsim_state *s);

// complex128 fused blocks of 4 qubits (fused64.cu): bytes of one block's
// slot (W digit planes + column exponents), kernel set-up (grid), the build
// of nb blocks' slots from their gate lists (block-local gates, 72 bytes
// each, offsets goff[0..nb]), and one block's apply
size_t fused_c128_slot_bytes();
int fused_c128_prepare(qsim_state *s, int *grid);
int launch_fuse_build_c128(qsim_state *s, const void *gates, const int *goff, int nb, void *out);
int launch_fused_c128(qsim_state *s, const void *block, const int *pos, int grid);
int launch_probabilities(qsim_state *s, void *dev_out, int out_real);
int launch_collapse(qsim_state *s, int qubit, int outcome, double scale);
int run_sample(qsim_state *s, uint64_t shots, uint64_t seed, uint64_t *out, int out_on_device,
               double *norm_out = nullptr, double *expz_out = nullptr);
// whether run_sample can form <sum Z> in its sub-block pass (complex64, n >= 13)
bool sample_observe_fused(const qsim_state *s);

// ---------------------------------------------------------------- plan lowering
// A circuit gate reduced to what the tile and block planners need: a 2x2
// matrix on one target with a set of control qubits.  SWAP is lowered to
// three CNOT-type moves; identity gates are dropped.
struct SGate {
    int op;              // GateOp (no OP_SWAP / OP_IDENTITY here)
    int target;
    uint64_t ctrl;       // control qubits
    double m[8];
    int orig;            // index of the circuit gate it comes from (OP_SUPER: index of its 4 x 4 matrix)
    int target2 = -1;    // OP_SUPER: the second qubit (above target)
    uint64_t xq() const
    {
        if (op == OP_SUPER) return (1ull << target) | (1ull << target2);
        return (op == OP_DENSE || op == OP_ANTIDIAG || op == OP_XPERM) ? (1ull << target) : 0ull;
    }
    uint64_t dq() const { return ctrl | ((op == OP_DIAG || op == OP_DIAG_HI) ? (1ull << target) : 0ull); }
};

// true when the two gates commute: every shared qubit is acted on diagonally by both
bool commute(const SGate &a, const SGate &b);
void lower_gates(const sim_gate *gates, size_t n_gates, std::vector<SGate> *out);

// one lowered gate (up to 3 controls) as its own per-gate launch
int launch_sgate(qsim_state *s, const SGate &g);

// ---------------------------------------------------------------- staged / fused plans
int apply_circuit_staged(qsim_state *s, const sim_gate *gates, size_t n_gates, const sim_plan_opts &o);
int apply_circuit_fused(qsim_state *s, const sim_gate *gates, size_t n_gates, const sim_plan_opts &o);
// fused blocks of k qubits over lowered gates that may hold OP_SUPER entries
// (a density matrix's channels; sup = their 4 x 4 matrices, 32 doubles each,
// row-major (re, im), indexed by SGate::orig)
int apply_sgates_fused(qsim_state *s, const std::vector<SGate> &g, const double *sup, int k);
int apply_circuit_learned(qsim_state *s, const sim_gate *gates, size_t n_gates, const sim_plan_opts &o);
int plan_features(int n, int dtype, const sim_gate *gates, size_t n_gates, int v, float *out);
// the learned plan's variant per window for a complex64 register with a cost
// model (also stored as the handle's last plan)
int learned_choose(qsim_state *s, const sim_gate *gates, size_t n_gates, std::vector<int> *best);
// blocks of the fused plan (depth 0 = the depth the plan runs with) and, when
// passes_out is given, the passes over the state (multi-block passes pair
// blocks when multi is set)
int describe_fused(int n, const sim_gate *gates, size_t n_gates, int k, int64_t *blocks_out, int depth = 0,
                   bool multi = true, int64_t *passes_out = nullptr);
// the (cheaper) planner depth the learned plan's features are computed with
int fused_feature_depth();
int describe_staged(int n, int dtype, const sim_gate *gates, size_t n_gates, int tile_qubits, int64_t *passes,
                    int64_t *ops, int64_t *layout_changes, int32_t *order, size_t order_cap, size_t *order_len);
int encode_staged(int n, int dtype, const sim_gate *gates, size_t n_gates, int tile_qubits, sim_tile_op *ops,
                  size_t ops_cap, int32_t *info, size_t info_cap, size_t *n_ops, size_t *n_passes);

// f(0) .. f(count - 1) on up to 16 host threads: the calling thread and a
// persistent pool (pool.cu).  Serial for one index, inside a pool thread, or
// on a one-core host.  The calling thread can finish any call alone.
void parallel_run(size_t count, void (*fn)(void *, size_t), void *ctx);
template <typename F>
void parallel_for(size_t count, F f)
{
    parallel_run(count, [](void *c, size_t i) { (*static_cast<F *>(c))(i); }, &f);
}

// host-side SplitMix64 draw (Steele, Lea & Flood 2014)
uint64_t splitmix64_host(uint64_t x);
double uniform_host(uint64_t seed, uint64_t s);

// grow a device buffer owned by the handle (stream-ordered)
int ensure_device(qsim_state *s, void **buf, size_t *cap, size_t need);
int ensure_host_pinned(void **buf, size_t *cap, size_t need);

}  // namespace qsim
