/*
 * qsim_gb300.h -- C ABI of the GB300 (sm_103a) dense state-vector simulator.
 *
 * The operations are those of Kelly, "Simulating Quantum Computers Using
 * OpenCL" (arXiv:1805.00988): a register of n qubits held as 2^n complex
 * amplitudes (§2.1), single-qubit gates given as 2x2 matrices applied by
 * Algorithm 1 (§2.3), the same gates with control qubits (§2.3, App. B.2),
 * probabilities |a_j|^2 (App. B.3) and measurement / repeated sampling from
 * one state (§1.3.3, §2.4).
 *
 * Conventions used by every entry point:
 *   - amplitude j is the coefficient of basis state |j>; qubit t is bit t of
 *     j (qubit 0 = least-significant bit), as the App. B kernels index it.
 *   - SIM_C64 = interleaved (re, im) FP32 pairs, 8 bytes per amplitude (§2.1);
 *     SIM_C128 = interleaved FP64 pairs, 16 bytes.
 *   - a gate matrix is [[A, B], [C, D]] given as 8 doubles
 *     (A.re, A.im, B.re, B.im, C.re, C.im, D.re, D.im), row-major (App. B.1).
 *     A controlled gate updates only index pairs whose control bits are all 1.
 *   - all sizes are in elements unless named *_bytes.
 *
 * Ownership and ordering: host arrays passed in are copied before the call
 * returns.  Work is enqueued on the handle's CUDA stream and is asynchronous
 * unless the entry point returns a host value (it then synchronises that
 * stream).  Device pointers passed in stay owned by the caller.  A handle
 * (state, batch or cost model) is used by one host thread at a time; distinct
 * handles may be used from different threads.
 *
 * Errors: every entry point returns a sim_status; nothing throws or aborts
 * across the ABI.  Arguments are validated on the host before any launch.
 * sim_last_error() returns a thread-local message for the last failure.
 */
#ifndef QSIM_GB300_H
#define QSIM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qsim_state *sim_t;

typedef enum { SIM_C64 = 0, SIM_C128 = 1 } sim_dtype;
typedef enum { SIM_F32 = 0, SIM_F64 = 1 } sim_real;

typedef enum {
    SIM_OK = 0,
    SIM_EINVAL = 1,        /* bad argument (qubit out of range, duplicate control, ...) */
    SIM_ENOMEM = 2,        /* device allocation failed or state does not fit */
    SIM_ECUDA = 3,         /* a CUDA runtime call failed */
    SIM_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    SIM_EUNSUPPORTED = 5   /* valid request this build does not implement */
} sim_status;

/* Gate kinds of sim_gate.kind.  SIM_GATE_U takes its matrix from
 * sim_gate.matrix; the named kinds build it from sim_gate.params:
 *   RX/RY/RZ(theta) = exp(-i theta sigma / 2), P(lambda) = diag(1, e^{i lambda}),
 *   U3(theta, phi, lambda) = [[cos t/2, -e^{i l} sin t/2], [e^{i p} sin t/2, e^{i(p+l)} cos t/2]].
 * SIM_GATE_SWAP exchanges qubits target and target2. */
typedef enum {
    SIM_GATE_U = 0, SIM_GATE_X = 1, SIM_GATE_Y = 2, SIM_GATE_Z = 3, SIM_GATE_H = 4,
    SIM_GATE_S = 5, SIM_GATE_SDG = 6, SIM_GATE_T = 7, SIM_GATE_TDG = 8,
    SIM_GATE_RX = 9, SIM_GATE_RY = 10, SIM_GATE_RZ = 11, SIM_GATE_P = 12, SIM_GATE_U3 = 13,
    SIM_GATE_SWAP = 14,
    /* noise channels, for sim_dm_apply_circuit only: on qubit target, no
     * controls, parameter params[0] in [0, 1] (see sim_channel_kind) */
    SIM_GATE_CH_DEPOLARIZING = 16, SIM_GATE_CH_AMPLITUDE_DAMPING = 17, SIM_GATE_CH_PHASE_DAMPING = 18,
    SIM_GATE_CH_BIT_FLIP = 19, SIM_GATE_CH_PHASE_FLIP = 20
} sim_gate_kind;

/* One gate of a circuit (112 bytes, no padding). */
typedef struct sim_gate {
    int32_t kind;          /* sim_gate_kind */
    int32_t target;        /* target qubit */
    int32_t target2;       /* second qubit of SIM_GATE_SWAP, else ignored */
    int32_t n_controls;    /* 0, 1 or 2 */
    int32_t controls[2];   /* control qubits; all must be 1 for the update */
    double params[3];      /* theta, phi, lambda */
    double matrix[8];      /* SIM_GATE_U: A, B, C, D as (re, im) */
} sim_gate;

/* How sim_apply_circuit schedules a gate list.  Every plan computes the same
 * product of gates (Algorithm 1 applied gate after gate); they differ in how
 * many passes over the state they make. */
typedef enum {
    SIM_PLAN_PER_GATE = 0,   /* one kernel launch per gate (one state pass each) */
    SIM_PLAN_STAGED = 1,     /* runs of gates applied per tile in one pass (registers + shared memory) */
    SIM_PLAN_FUSED = 2,      /* gates fused into k-qubit unitaries built in FP64, applied on tensor cores */
    SIM_PLAN_LEARNED = 3     /* per-window (or whole-circuit) variant chosen by the trained cost model */
} sim_plan_kind;

typedef struct sim_plan_opts {
    int32_t plan;            /* sim_plan_kind */
    int32_t fuse_k;          /* SIM_PLAN_FUSED: qubits per fused block.  complex64: 3..6 (0 = 5);
                                k <= 5 runs 3xTF32, k = 6 an FP16 hi / lo split (same 22
                                significant bits) of operands scaled by powers of two: the state by
                                one chosen from its norm (one extra pass over the state per call),
                                each block's matrix by one chosen from the product of its gates'
                                spectral norms, so states of any magnitude are applied at the same
                                precision relative to their norm; SIM_EUNSUPPORTED if that product
                                exceeds 2^114.  complex128: 4 only (0 = 4): rows and columns are
                                written in 47-bit fixed point relative to their largest entry, cut
                                into six balanced 8-bit integer digits, and the digit products are
                                summed exactly on the FP16 tensor cores (error-free splitting of
                                Ozaki, Ogita, Oishi and Rump 2012); each result is within about
                                2^-42 of its row's and column's largest entries at worst (2^-47 for
                                the fixed-point rounding).  Every fused plan needs
                                n >= k + 7 (SIM_EINVAL otherwise). */
    int32_t tile_qubits;     /* SIM_PLAN_STAGED: tile size log2 (0 = default) */
    int32_t flags;           /* SIM_FLAG_* bits, 0 = defaults */
} sim_plan_opts;

/* SIM_PLAN_FUSED, k = 5: apply each pair of consecutive blocks whose qubits
 * (with qubit 0) fit one 12-qubit tile in a single pass over the state (the
 * tile stays in shared memory between the two blocks).  Off by default: on
 * this GPU the pass costs more than two single-block passes (the per-tile
 * chain convert -> MMA -> write-back -> convert -> MMA runs serially). */
#define SIM_FLAG_MULTI_BLOCK_PASSES 1

/* ---- handles --------------------------------------------------------------
 * sim_create: allocate a 2^n state on the current CUDA device and set it to
 *   |0...0> (§2.1).  n in [1, 34]; the state must fit in free device memory
 *   (SIM_ENOMEM otherwise).  stream: a cudaStream_t (NULL = the handle
 *   creates its own non-blocking stream; pass cudaStreamLegacy to work on
 *   the legacy default stream).
 * sim_create_from_buffer: wrap caller-owned device memory of at least
 *   2^n * sizeof(amplitude) bytes, 16-byte aligned; its contents are kept.
 * sim_destroy: free what the handle owns (not a wrapped buffer).
 * The first handle created on a device sets that device's L2 fetch
 * granularity hint for this process's CUDA context to 64 bytes
 * (cudaLimitMaxL2FetchGranularity; it ends with the process): gates whose
 * lowest control or target is qubit 3 touch 64-byte runs, and with the
 * default the memory system fetched the unused half of every 128-byte line. */
int sim_create(int n, int dtype, void *stream, sim_t *out);
int sim_create_from_buffer(int n, int dtype, void *dev_ptr, size_t bytes, void *stream, sim_t *out);
int sim_destroy(sim_t s);
int sim_state_info(sim_t s, int *n, int *dtype, void **dev_ptr, size_t *bytes);
int sim_synchronize(sim_t s);

/* sim_set_basis_state: the state becomes |j>, j < 2^n (§2.1 starts at j = 0). */
int sim_set_basis_state(sim_t s, uint64_t j);

/* sim_load_state / sim_copy_state: copy 2^n amplitudes of the handle's dtype
 * from / to src / dst (host memory when *_is_host, else device memory). */
int sim_load_state(sim_t s, const void *src, int src_is_host);
int sim_copy_state(sim_t s, void *dst, int dst_is_host);

/* ---- gates ----------------------------------------------------------------
 * sim_apply_gate: Algorithm 1 (§2.3) with matrix U on qubit target; with
 *   n_controls in {1, 2} only the pairs whose control bits are all 1 are
 *   updated (§2.3, App. B.2).  SIM_EINVAL if a qubit is out of range, a
 *   control equals the target or two controls are equal.
 * sim_apply_circuit: apply n_gates gates in order, scheduled by opts (NULL =
 *   SIM_PLAN_PER_GATE).  The whole list is validated before anything runs. */
int sim_apply_gate(sim_t s, const double U[8], int target, const int *controls, int n_controls);
int sim_apply_circuit(sim_t s, const sim_gate *gates, size_t n_gates, const sim_plan_opts *opts);

/* ---- measurement ------------------------------------------------------------
 * sim_probabilities: p_j = |a_j|^2 for all j (App. B.3) into dev_out, a device
 *   array of 2^n floats (out_real = SIM_F32) or doubles (SIM_F64).
 * sim_norm: sum_j |a_j|^2 accumulated in FP64 (complex128: squares in FP64;
 *   complex64: exact FP32 squares summed with compensation in chunks of 8
 *   amplitudes, each carried into FP64; within about 1e-12 relative of the
 *   exact sum).
 * sim_measure: measure one qubit in the computational basis (§1.3.3):
 *   p0, p1 summed in FP64 (accumulated as for sim_norm); outcome 0 iff
 *   p0 > u (p0 + p1) with
 *   u = (splitmix64(seed + draw) >> 11) * 2^-53 (SplitMix64, Steele et al.
 *   2014); the other half is zeroed and the kept half scaled by
 *   1 / sqrt(p_outcome).  *prob (may be NULL) gets p_outcome / (p0 + p1).
 * sim_sample: non-destructive shot sampling (§2.4): shot s is the smallest j
 *   with C_j > u_s C_total, C the inclusive FP64 prefix of |a_j|^2 (partial
 *   sums accumulated as for sim_norm; a shot whose target lies within about
 *   1e-12 C_total of a prefix value may land on the neighbouring index, and
 *   an amplitude that is exactly zero is never drawn),
 *   u_s = (splitmix64(seed + s) >> 11) * 2^-53.  out: shots uint64 indices,
 *   on the device when out_on_device, else host memory.
 * sim_expect_z_sum: <sum_i Z_i> = sum_x |a_x|^2 (n - 2 popcount x), FP64
 *   (complex64: squares accumulated as for sim_norm, weighted by exact
 *   products).
 * sim_norm_expect_z: sim_norm and sim_expect_z_sum from one pass over the
 *   state (both read every |a_x|^2; the norm is the unweighted sum of the
 *   same accumulators, within about 1e-12 relative of sim_norm's).
 * sim_sample_observe: sim_sample, plus the norm and <sum_i Z_i> of the same
 *   state.  complex64 from 13 qubits, with shots > 0: one pass over the state
 *   gives the sampler's sub-block sums, their total (the norm, C_total) and
 *   the popcount-weighted sum; the shots are the ones sim_sample draws for
 *   the same seed.  Otherwise sim_norm_expect_z's pass runs first.  norm and
 *   expz are host pointers (required); out as for sim_sample. */
int sim_probabilities(sim_t s, void *dev_out, int out_real);
int sim_norm(sim_t s, double *out);
int sim_measure(sim_t s, int qubit, uint64_t seed, uint64_t draw, int *outcome, double *prob);
int sim_sample(sim_t s, uint64_t shots, uint64_t seed, uint64_t *out, int out_on_device);
int sim_expect_z_sum(sim_t s, double *out);
int sim_norm_expect_z(sim_t s, double *norm, double *expz);
int sim_sample_observe(sim_t s, uint64_t shots, uint64_t seed, uint64_t *out, int out_on_device, double *norm,
                       double *expz);

/* ---- density matrices and noise ---------------------------------------------
 * The paper names density matrices among a simulator's outputs (§1) without
 * a method; these calls give them the operations the paper defines for a
 * state (§1.3.3, §2.3, §2.4).  A density-matrix handle holds rho of n qubits
 * (n in [1, 17]) as a register of 2n qubits: rho[r][c] is amplitude
 * (r << n) | c (4^n amplitudes of the handle's dtype; sim_copy_state /
 * sim_load_state move them in that order, sim_state_info reports 2n).  The
 * state-vector calls that would read it as a state (sim_apply_gate,
 * sim_apply_circuit, sim_set_basis_state, sim_probabilities, sim_norm,
 * sim_measure, sim_sample, sim_expect_z_sum) return SIM_EINVAL on it, and the
 * sim_dm_* calls SIM_EINVAL on a state-vector handle.
 *
 * Channels (Nielsen & Chuang §8.3), p in [0, 1]:
 *   DEPOLARIZING      rho -> (1 - p) rho + p I / 2 (Kraus sqrt(1 - 3p/4) I,
 *                     sqrt(p/4) X, Y, Z)
 *   AMPLITUDE_DAMPING diag(1, sqrt(1 - p)), sqrt(p) |0><1|
 *   PHASE_DAMPING     diag(1, sqrt(1 - p)), sqrt(p) |1><1|
 *   BIT_FLIP          sqrt(1 - p) I, sqrt(p) X
 *   PHASE_FLIP        sqrt(1 - p) I, sqrt(p) Z
 *
 * sim_dm_create / sim_dm_create_from_buffer: as sim_create /
 *   sim_create_from_buffer for the 2n-qubit register (sim_dm_create starts in
 *   |0...0><0...0|; a wrapped buffer keeps its contents).
 * sim_dm_info: *n = the number of qubits of rho.
 * sim_dm_set_basis_state: rho = |j><j|.
 * sim_dm_set_pure: rho = |psi><psi| from state-vector handle psi (n qubits,
 *   same dtype; ordered after psi's pending work).
 * sim_dm_apply_circuit: for each gate G on qubit t, rho -> G rho G^dagger
 *   (G on register qubit t + n, conj(G) on register qubit t, controls
 *   likewise), scheduled by opts like sim_apply_circuit on the register; a
 *   channel kind (SIM_GATE_CH_*) applies that channel where it stands (one
 *   pass over the register).
 * sim_channel_kraus: the Kraus operators of SIM_CHANNEL_* kind with
 *   parameter p into kraus (host, up to 4 x 8 doubles, each a 2x2 matrix laid
 *   out as sim_apply_gate's U); *n_kraus gets their count.
 * sim_dm_apply_kraus: rho -> sum_m K_m rho K_m^dagger on qubit target,
 *   n_kraus in [1, 16] matrices of 8 doubles (host); the map need not be
 *   trace preserving.  sim_dm_apply_channel: the same for a named channel.
 * sim_dm_probabilities: p_j = Re rho[j][j] into a device array of 2^n floats
 *   (out_real = SIM_F32) or doubles.
 * sim_dm_trace: sum_j Re rho[j][j] in FP64.  sim_dm_purity: sum |rho_rc|^2
 *   (= tr rho^2 for Hermitian rho), accumulated as sim_norm.
 * sim_dm_expect_z_sum: sum_j Re rho[j][j] (n - 2 popcount j), FP64.
 * sim_dm_measure: measure qubit q as sim_measure does on a state: p0, p1
 *   from the diagonal, the outcome from the same draw, then
 *   rho -> P rho P / p(outcome), P the projector on bit q = outcome.
 * sim_dm_sample: shots from p_j as sim_sample draws them from |a_j|^2 (rho
 *   unchanged).
 * Trace, <sum Z>, measurement and sampling read p_j through FP64 square roots
 *   sqrt(max(p_j, 0)) whose squares they sum (within an FP64 rounding of p_j);
 *   a diagonal entry below zero, which only rounding produces for a physical
 *   rho, counts as zero there. */
typedef enum {
    SIM_CHANNEL_DEPOLARIZING = 0, SIM_CHANNEL_AMPLITUDE_DAMPING = 1, SIM_CHANNEL_PHASE_DAMPING = 2,
    SIM_CHANNEL_BIT_FLIP = 3, SIM_CHANNEL_PHASE_FLIP = 4
} sim_channel_kind;
int sim_dm_create(int n, int dtype, void *stream, sim_t *out);
int sim_dm_create_from_buffer(int n, int dtype, void *dev_ptr, size_t bytes, void *stream, sim_t *out);
int sim_dm_info(sim_t s, int *n);
int sim_dm_set_basis_state(sim_t s, uint64_t j);
int sim_dm_set_pure(sim_t s, sim_t psi);
int sim_dm_apply_circuit(sim_t s, const sim_gate *gates, size_t n_gates, const sim_plan_opts *opts);
int sim_channel_kraus(int kind, double p, double *kraus, int *n_kraus);
int sim_dm_apply_kraus(sim_t s, int target, const double *kraus, int n_kraus);
int sim_dm_apply_channel(sim_t s, int kind, double p, int target);
int sim_dm_probabilities(sim_t s, void *dev_out, int out_real);
int sim_dm_trace(sim_t s, double *out);
int sim_dm_purity(sim_t s, double *out);
int sim_dm_expect_z_sum(sim_t s, double *out);
int sim_dm_measure(sim_t s, int qubit, uint64_t seed, uint64_t draw, int *outcome, double *prob);
int sim_dm_sample(sim_t s, uint64_t shots, uint64_t seed, uint64_t *out, int out_on_device);

/* ---- batches of small circuits ---------------------------------------------
 * Many independent registers, each started in |0...0> (§2.1), each with its
 * own gate list applied by Algorithm 1 (§2.3), each returning
 * <sum_i Z_i> = sum_x |a_x|^2 (n - 2 popcount x) (FP64 accumulation).
 *
 * sim_batch_create: plan and upload `count` circuits (complex64 states).
 *   n_qubits[c] in [1, 24]; the gates of circuit c are
 *   gates[gate_offsets[c] .. gate_offsets[c+1]) (count + 1 offsets, non-
 *   decreasing).  All host arrays are copied.  The run is captured once as a
 *   CUDA graph (a reset kernel + one persistent kernel with a device work
 *   queue); stream as in sim_create.  SIM_EINVAL for invalid circuits,
 *   SIM_ENOMEM if the scratch (one state per circuit above 13 qubits, 8 B per
 *   amplitude, plus plan data) does not fit.
 * sim_batch_run: launch the graph; expz_out gets `count` doubles (device
 *   memory when out_on_device, else host memory); synchronises the stream.
 *   SIM_ETIMEOUT if a bounded device-side wait gave up (about one second);
 *   the CUDA context stays usable.
 * sim_batch_info: items in the work queue, passes, encoded ops, device bytes
 *   held, persistent grid size (any output may be NULL).
 * sim_batch_destroy: release everything the batch holds. */
typedef struct qsim_batch *sim_batch_t;
int sim_batch_create(int count, const int32_t *n_qubits, const int64_t *gate_offsets, const sim_gate *gates,
                     void *stream, sim_batch_t *out);
/* sim_batch_create_opts: as sim_batch_create, with the launch configuration
 *   (no paper counterpart; the autotuner picks it per workload):
 *   tile_qubits in {0, 11, 12, 13} (0 = 13): qubits per register tile (a
 *   circuit of up to that many qubits lives in one CTA; larger ones run tile
 *   passes over a scratch state); ctas_per_sm >= 0 (0 = as many as fit: two
 *   with 13-qubit tiles, three with 11 or 12): persistent CTAs per SM.
 *   SIM_EINVAL outside those ranges or above what fits.
 * sim_batch_config: the configuration a batch uses, its algorithmic flops
 *   (8 per complex multiply-add of the gates as given, summed over the
 *   circuits) and the scratch-state bytes its plan must read and write per
 *   run (any output may be NULL). */
typedef struct sim_batch_opts {
    int32_t tile_qubits;
    int32_t ctas_per_sm;
    int32_t reserved[2];     /* 0 */
} sim_batch_opts;
int sim_batch_create_opts(int count, const int32_t *n_qubits, const int64_t *gate_offsets, const sim_gate *gates,
                          const sim_batch_opts *opts, void *stream, sim_batch_t *out);
int sim_batch_config(sim_batch_t b, sim_batch_opts *used, double *alg_flops, double *alg_scratch_bytes);
int sim_batch_run(sim_batch_t b, double *expz_out, int out_on_device);
int sim_batch_info(sim_batch_t b, int64_t *items, int64_t *passes, int64_t *ops, int64_t *scratch_bytes, int *grid);
int sim_batch_destroy(sim_batch_t b);

/* ---- plan cost model ---------------------------------------------------------
 * A small MLP (d_in -> hidden -> hidden -> 1, ReLU) trained on the GPU by the
 * library's own forward / backward / Adam kernels to predict the log of a
 * circuit segment's run time under each plan variant, up to an additive
 * constant per register size (only the variants of one segment are
 * compared with each other; there is no paper
 * counterpart: the paper applies every gate with its own kernel launch).
 * Parameters: one FP32 vector W1 (d_in x hidden, row-major), b1, W2, b2,
 * W3 (hidden x 1), b3 -- sim_mlp_param_count() floats.
 *
 * sim_mlp_create: zero parameters; d_in, hidden in [1, 256]; stream as in
 *   sim_create.
 * sim_mlp_set_params / get_params: host arrays of sim_mlp_param_count floats
 *   (set also clears the Adam moments).
 * sim_mlp_forward: y[r] for rows r of x (rows x d_in, row-major); x and y
 *   device pointers when on_device, else host.
 * sim_mlp_loss_grad: L = mean (y - t)^2 and dL/dparams (host, may be NULL).
 * sim_mlp_train: `steps` full-batch Adam steps (beta1 0.9, beta2 0.999,
 *   eps 1e-8, learning rate lr); *final_loss (may be NULL) after the last.
 * sim_set_cost_model: SIM_PLAN_LEARNED on this handle consults model m (NULL
 *   = no model: the greedy fixed-k plan is used).  The model must outlive the
 *   handle's use of it.  A complex128 handle runs SIM_PLAN_LEARNED without
 *   consulting the model (trained on complex64 timings): as the fused plan
 *   with k = 4 when n >= 11 (tensor-core digit products; the per-gate and
 *   register-tile kernels are bound by the FP64 pipe), else per gate. */
typedef struct qsim_mlp *sim_mlp_t;
int sim_mlp_param_count(int d_in, int hidden);
int sim_mlp_create(int d_in, int hidden, void *stream, sim_mlp_t *out);
int sim_mlp_destroy(sim_mlp_t m);
int sim_mlp_set_params(sim_mlp_t m, const float *params);
int sim_mlp_get_params(sim_mlp_t m, float *params);
int sim_mlp_forward(sim_mlp_t m, const float *x, int64_t rows, float *y, int on_device);
int sim_mlp_loss_grad(sim_mlp_t m, const float *x, const float *t, int64_t rows, int on_device, float *loss,
                      float *grad);
int sim_mlp_train(sim_mlp_t m, const float *x, const float *t, int64_t rows, int steps, float lr, int on_device,
                  float *final_loss);
int sim_set_cost_model(sim_t s, sim_mlp_t m);

/* sim_plan_features: the cost model's input row for a segment of gates on an
 *   n-qubit register under plan variant v (0 per-gate, 1 staged 12-qubit
 *   tiles, 2 staged 13-qubit tiles, 3..6 fused with k = 3..6): SIM_FEATURES
 *   floats into out.  Host only. */
#define SIM_FEATURES 16
#define SIM_VARIANTS 7
int sim_plan_features(int n, int dtype, const sim_gate *gates, size_t n_gates, int variant, float *out);
/* sim_last_plan: the variant the last SIM_PLAN_LEARNED call chose for each
 *   window of gates (up to cap entries; the count in *len). */
int sim_last_plan(sim_t s, int32_t *variants, size_t cap, size_t *len);

/* ---- plan introspection (host only, no GPU needed) ---------------------------
 * sim_plan_describe: build the SIM_PLAN_STAGED schedule of a circuit for an
 *   n-qubit register of the given dtype without running it.  Outputs (any may
 *   be NULL): the number of tile passes, of ops (gate ops, layout changes,
 *   and phase ramps -- one per ramp, whatever its records), of register-layout
 *   changes, and the order in which the gates are applied (circuit indices;
 *   a SWAP appears three times, lowered to three CNOT-type moves; identity
 *   gates are dropped) -- up to order_cap entries, the full length in
 *   *order_len.  SIM_EINVAL if no tile fits (n below 11) or a gate is invalid.
 *   With opts->plan = SIM_PLAN_FUSED (fuse_k 0 = 5): *passes gets the passes
 *   the fused plan makes over the state (a multi-block pass counts once,
 *   see SIM_FLAG_MULTI_BLOCK_PASSES),
 *   *ops the fused blocks; *layout_changes and *order_len are set to 0.
 *   Other plans: SIM_EUNSUPPORTED. */
int sim_plan_describe(int n, int dtype, const sim_gate *gates, size_t n_gates, const sim_plan_opts *opts,
                      int64_t *passes, int64_t *ops, int64_t *layout_changes, int32_t *order, size_t order_cap,
                      size_t *order_len);

/* sim_plan_staged_ops: the SIM_PLAN_STAGED encoding of a circuit, host only,
 *   for inspection and for checking the planner without a GPU (the record
 *   layout follows the library's version).  A tile is 2^M amplitudes: local
 *   bits 0..4 are qubits 0..4, local bit 5 + i is the pass's high qubit i;
 *   256 threads hold 2^(M - 8) registers each.  Register layout l places
 *   register bit j and thread bit i on local bits given by the library's
 *   layout tables (layout 0: the I/O layout).  Each record: kind (0 layout
 *   change to arg, 1 dense / 2 antidiagonal / 3 exchange 2 x 2 on register
 *   bit arg, 4 diagonal diag(a, d), 5 phase d on |1>, 6 sign flip, 7 phase
 *   ramp, 8 no-op), the conditions thr_c / out_c / km_c (thread bits, outer
 *   qubits, registers that satisfy the controls; plain = no condition), the
 *   target of a diagonal op or a ramp's shared qubit as thr_t / out_t / km_t,
 *   and the coefficients m = (A, B, C, D) as (re, im) pairs (a ramp's tables
 *   span its records' m, four complex entries per record: entry k < 2^RB is
 *   register k's factor, 2^RB + x and 2^RB + 16 + y the factors of thread
 *   bits 0..3 set in x and 4..7 set in y).  ops: up to ops_cap records;
 *   info: SIM_TILE_PASS_INFO int32 per pass (first record, record count, M,
 *   register bits, amplitudes per I/O vector, number of high qubits, the
 *   high qubits); *n_ops, *n_passes the full counts.  SIM_EINVAL if no tile
 *   fits or a gate is invalid. */
typedef struct sim_tile_op {
    int32_t kind;
    int32_t arg;
    uint32_t thr_c;
    int32_t plain;
    uint64_t out_c;
    uint64_t km_c;
    uint64_t km_t;
    uint32_t thr_t;
    uint32_t pad;
    uint64_t out_t;
    double m[8];
} sim_tile_op;
#define SIM_TILE_PASS_INFO 24
int sim_plan_staged_ops(int n, int dtype, const sim_gate *gates, size_t n_gates, int tile_qubits, sim_tile_op *ops,
                        size_t ops_cap, int32_t *info, size_t info_cap, size_t *n_ops, size_t *n_passes);

/* ---- instrumentation --------------------------------------------------------
 * sim_profile_enable: when on, every kernel launch of the handle is bracketed
 *   by CUDA events on the handle's stream.
 * sim_profile_read: synchronise, then report per kernel class (see
 *   sim_kernel_class_name) the launches, summed device milliseconds and
 *   summed algorithmic bytes (the state bytes each launch must read and
 *   write: 2S / 2^c for a dense gate with c controls, S for a pass over the
 *   whole state, ...) and summed algorithmic flops (8 per complex multiply-
 *   add of the gate arithmetic; 3 real GEMMs per fused block) since the last
 *   reset; any output array may be NULL;
 *   reset != 0 clears the counters.  Fills at most max_classes entries.
 * sim_launch_count: kernels this handle has launched since creation. */
int sim_profile_enable(sim_t s, int on);
int sim_profile_read(sim_t s, int max_classes, uint64_t *launches, double *total_ms, double *alg_bytes,
                     double *alg_flops,
                     int reset);
int sim_launch_count(sim_t s, uint64_t *out);
const char *sim_kernel_class_name(int k);
int sim_num_kernel_classes(void);

/* sim_measure_fma_peak: measured FMA throughput of the current device in
 *   TFLOP/s (2 flops per FMA) -- which = 0: FP32 fma, 1: packed FP32
 *   fma.rn.f32x2, 2: FP64 fma.  A few milliseconds of GPU work on the legacy
 *   default stream; synchronises.  Used as the arithmetic roofline of kernels
 *   that are not bound by HBM. */
int sim_measure_fma_peak(int which, double *tflops);

/* sim_norm_noalloc: sum_j |a_j|^2 in FP64 of a caller's state -- 2^n
 *   amplitudes of dtype at dev_state (device memory, 16-byte aligned) --
 *   enqueued on `stream` (NULL = the legacy default stream); the result goes to
 *   *out (host memory) and the call synchronises that stream.  The paper has
 *   no counterpart of this entry point: it exists for callers that cannot
 *   allocate device memory when they need a norm (for example while another
 *   allocator, such as a framework's caching allocator or a memory pool sized
 *   to the whole GPU, holds all free device memory, or where entering the
 *   device allocator, which can synchronise the device, is not acceptable).
 *   It allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 *   routine.  Its only scratch is a fixed 1217-double (9,736-byte) array
 *   compiled into the library, which every GPU that loads the library holds
 *   until the process exits.  All calls share that array: calls that overlap
 *   on the GPU race and must be serialised by the caller; each call overwrites
 *   every slot it reads, so nothing needs clearing between calls.  The first
 *   call on a device looks up the array's device address (once per device,
 *   with that device current); make that first call before any stream
 *   capture.  n must be in [1, 34] (SIM_EINVAL beyond, with a message). */
int sim_norm_noalloc(const void *dev_state, int n, int dtype, void *stream, double *out);

/* Thread-local description of the last failure (empty string if none). */
const char *sim_last_error(void);
/* Library version string. */
const char *sim_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QSIM_GB300_H */
