// batch.cu -- many small circuits of uneven qubit counts in one persistent
// launch, captured in a CUDA graph, returning <sum_i Z_i> per circuit.
//
// Every circuit is planned on the host like the staged plan (M-qubit tiles,
// M = 11, 12 or 13 per batch, chosen by the caller or the autotuner; gates
// encoded per pass; adjacent single-qubit gates on the same qubit are merged
// into one 2x2 first).  A circuit of at most M qubits is one tile: it lives in
// the registers of one CTA from |0...0> to <Z> and never touches global
// memory.  A larger circuit keeps its state in a scratch buffer and runs pass
// after pass, each pass split into tiles.
//
// The launch is persistent: as many CTAs as fit on the GPU at once, each
// taking work items (circuit, pass, tile) from a device queue in a host-built
// order (all first passes, then all second passes, ...).  A tile of pass p > 0
// waits until every tile of pass p - 1 of its circuit has been stored; those
// items were handed out earlier to CTAs that are running, so the wait always
// ends.  It is bounded all the same (about one second of %globaltimer): on a
// timeout the CTA records SIM_ETIMEOUT in a status word and every CTA leaves
// the queue.  The last tile of a circuit's last pass adds the per-tile partial
// sums of <sum Z> in a fixed order, so results are bit-reproducible.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "tile.cuh"

struct qsim_batch;

namespace qsim {

namespace {

constexpr int kBM = 13;                 // default tile qubits (complex64)
constexpr unsigned long long kWaitNs = 1000000000ull;

struct BCirc {
    int32_t n;            // qubits
    int32_t npass;
    int32_t ntiles;       // tiles per pass
    int32_t pad;
    int64_t pass0;        // first pass in the pass table
    int64_t part0;        // first partial-sum slot (ntiles of them)
    int64_t state0;       // first amplitude of its scratch state (multi-tile circuits)
};

struct BPass {
    int64_t op0;
    int32_t nops;
    int32_t need;         // tiles of the previous pass that must be stored first
    TileGeom geo;
};

struct BItem {
    int32_t circ, pass, tile, pad;
};

struct BCtl {             // device-side control block, zeroed before every run
    unsigned long long head;
    int status;
    int pad;
};

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__global__ void k_batch_reset(BCtl *ctl, int *done, int64_t ndone, int *finished, int64_t ncirc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (i == 0) { ctl->head = 0; ctl->status = 0; }
    for (int64_t j = i; j < ndone; j += stride) done[j] = 0;
    for (int64_t j = i; j < ncirc; j += stride) finished[j] = 0;
}

// tiles of up to 12 qubits fit three CTAs per SM (as the staged plan's),
// 13-qubit tiles two
template <int M>
__global__ void __launch_bounds__(kThr, M <= 12 ? 3 : 2)
    k_batch(float2 *__restrict__ scratch, const BCirc *__restrict__ circs, const BPass *__restrict__ passes,
            const StOp<float> *__restrict__ ops, const BItem *__restrict__ items, int64_t nitems, BCtl *ctl, int *done,
            int *finished, double *__restrict__ partial, double *__restrict__ out)
{
    constexpr int RB = M - kThrBits, RA = 1 << RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>(smem_raw);
    __shared__ long long cur;
    __shared__ int stop;
    __shared__ double red[kThr / 32];
    __shared__ int last;
    const int tid = threadIdx.x;

    for (;;) {
        if (tid == 0) {
            cur = (long long)atomicAdd(&ctl->head, 1ull);
            stop = (cur >= nitems) || (*reinterpret_cast<volatile int *>(&ctl->status) != 0);
        }
        __syncthreads();
        if (stop) break;
        const BItem it = items[cur];
        const BCirc c = circs[it.circ];
        const BPass &ps = passes[c.pass0 + it.pass];
        const bool single = c.ntiles == 1 && c.npass == 1 && c.n <= M;

        // wait for the previous pass of this circuit (bounded)
        if (it.pass > 0) {
            if (tid == 0) {
                volatile int *d = done + c.pass0 + it.pass - 1;
                const unsigned long long t0 = gtimer();
                while (*d < ps.need) {
                    if (*reinterpret_cast<volatile int *>(&ctl->status) != 0 || gtimer() - t0 > kWaitNs) {
                        atomicExch(&ctl->status, SIM_ETIMEOUT);
                        stop = 1;
                        break;
                    }
                    __nanosleep(200);
                }
                __threadfence();
            }
            __syncthreads();
            if (stop) break;
        }

        // tile base and I/O offsets (layout 0).  They are formed again after
        // the gate sequence from inputs the compiler cannot prove equal
        // instead of being held live across it (which spilled at two CTAs
        // per SM), as in the staged kernel.
        uint64_t base = 0;
        for (int i = 0; i < ps.geo.n_outer; ++i) base |= ((uint64_t)(it.tile >> i) & 1ull) << ps.geo.outer_pos[i];
        uint64_t toff, roff[RB];
        auto io_offsets = [&](const TileGeom &geo, int t, uint64_t b0) {
            toff = b0;
#pragma unroll
            for (int i = 0; i < kThrBits; ++i) {
                const int b = thr_local(M, RB, 2, 0, i);
                const uint64_t g = (b < kLow) ? (1ull << b) : (1ull << geo.hpos[b - kLow]);
                if ((t >> i) & 1) toff |= g;
            }
#pragma unroll
            for (int j = 0; j < RB; ++j) {
                const int b = reg_local(M, RB, 2, 0, j);
                roff[j] = (b < kLow) ? (1ull << b) : (1ull << geo.hpos[b - kLow]);
            }
        };
        io_offsets(ps.geo, tid, base);
        float *st = reinterpret_cast<float *>(scratch + c.state0);

        Regs<float, RA> v;
        if (it.pass == 0) {
            // |0...0>: amplitude 0 sits in register 0 of thread 0 of tile 0
#pragma unroll
            for (int p = 0; p < RA / 2; ++p) v.set2(p, 0.f, 0.f, 0.f, 0.f);
            if (base == 0 && tid == 0) v.setr(0, 1.f);
        } else {
#pragma unroll
            for (int k = 0; k < RA; k += 2) {
                uint64_t g = toff;
#pragma unroll
                for (int j = 1; j < RB; ++j)
                    if ((k >> j) & 1) g |= roff[j];
                const float4 t = __ldcg(reinterpret_cast<const float4 *>(st + 2 * g));
                v.set2(k >> 1, t.x, t.y, t.z, t.w);
            }
        }

        apply_ops<float, M>(v, ops + ps.op0, ps.nops, base, tid, sm,
                            reinterpret_cast<StOp<float> *>(smem_raw + ((size_t)1 << M) * 2 * sizeof(float)));
        {
            int t2 = tid;
            uint64_t b2 = base;
            const BPass *pp = passes + (c.pass0 + it.pass);
            asm volatile("" : "+r"(t2), "+l"(b2), "+l"(pp));
            io_offsets(pp->geo, t2, b2);
        }

        if (it.pass + 1 < c.npass) {
#pragma unroll
            for (int k = 0; k < RA; k += 2) {
                uint64_t g = toff;
#pragma unroll
                for (int j = 1; j < RB; ++j)
                    if ((k >> j) & 1) g |= roff[j];
                __stcg(reinterpret_cast<float4 *>(st + 2 * g),
                       make_float4(v.getr(k), v.geti(k), v.getr(k + 1), v.geti(k + 1)));
            }
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                atomicAdd(done + c.pass0 + it.pass, 1);
            }
        } else {
            // <sum Z> over this tile: |a_x|^2 (n - 2 popcount x), FP64
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < RA; ++k) {
                uint64_t g = toff;
#pragma unroll
                for (int j = 0; j < RB; ++j)
                    if ((k >> j) & 1) g |= roff[j];
                const double re = v.getr(k), im = v.geti(k);
                acc += (re * re + im * im) * (double)(c.n - 2 * __popcll(g));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if ((tid & 31) == 0) red[tid >> 5] = acc;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int w = 0; w < kThr / 32; ++w) s += red[w];
                if (single) {
                    out[it.circ] = s;
                    last = 0;
                } else {
                    partial[c.part0 + it.tile] = s;
                    __threadfence();
                    last = (atomicAdd(finished + it.circ, 1) == c.ntiles - 1);
                }
            }
            __syncthreads();
            if (last && tid == 0) {
                __threadfence();
                double s = 0.0;
                for (int t = 0; t < c.ntiles; ++t) s += *reinterpret_cast<volatile double *>(partial + c.part0 + t);
                out[it.circ] = s;
            }
        }
        __syncthreads();
    }
}

// merge runs of adjacent uncontrolled single-qubit gates on the same target
// into one 2x2 (FP64 product, later gate on the left)
void merge_single_qubit(std::vector<SGate> *g)
{
    std::vector<SGate> out;
    for (const SGate &s : *g) {
        if (!out.empty() && out.back().ctrl == 0 && s.ctrl == 0 && out.back().target == s.target) {
            SGate &b = out.back();
            double r[8];
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    double re = 0, im = 0;
                    for (int l = 0; l < 2; ++l) {
                        const double ar = s.m[2 * (2 * i + l)], ai = s.m[2 * (2 * i + l) + 1];
                        const double br = b.m[2 * (2 * l + j)], bi = b.m[2 * (2 * l + j) + 1];
                        re += ar * br - ai * bi;
                        im += ar * bi + ai * br;
                    }
                    r[2 * (2 * i + j)] = re;
                    r[2 * (2 * i + j) + 1] = im;
                }
            memcpy(b.m, r, sizeof r);
            b.op = classify_matrix(b.m);
            if (b.op == OP_IDENTITY) out.pop_back();
            continue;
        }
        out.push_back(s);
    }
    g->swap(out);
}

}  // namespace

}  // namespace qsim

using namespace qsim;

struct qsim_batch {
    int count = 0;
    int tile_qubits = kBM, ctas_per_sm = 0;
    double alg_flops = 0, alg_scratch_bytes = 0;
    cudaStream_t stream = nullptr;
    bool owns_stream = false;
    int grid = 0;
    int64_t nitems = 0, npasses = 0, nops = 0;
    size_t scratch_bytes = 0;
    void *dev = nullptr;              // one allocation for everything
    BCirc *circs = nullptr;
    BPass *passes = nullptr;
    StOp<float> *ops = nullptr;
    BItem *items = nullptr;
    BCtl *ctl = nullptr;
    int *done = nullptr, *finished = nullptr;
    double *partial = nullptr, *out = nullptr;
    float2 *scratch = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void batch_free(qsim_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->dev) cudaFree(b->dev);
    if (b->owns_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

namespace {

template <int M>
const void *batch_kernel() { return (const void *)k_batch<M>; }

const void *batch_kernel_for(int M)
{
    return M == 11 ? batch_kernel<11>() : M == 12 ? batch_kernel<12>() : batch_kernel<13>();
}

}  // namespace

extern "C" int sim_batch_create_opts(int count, const int32_t *n_qubits, const int64_t *gate_offsets,
                                     const sim_gate *gates, const sim_batch_opts *opts, void *stream,
                                     qsim_batch **out)
{
    set_error("");
    if (!out || count <= 0 || !n_qubits || !gate_offsets || (gate_offsets[count] > 0 && !gates))
        return fail(SIM_EINVAL, "sim_batch_create: bad arguments");
    *out = nullptr;
    const int M = (opts && opts->tile_qubits) ? opts->tile_qubits : kBM;
    const int want_per_sm = opts ? opts->ctas_per_sm : 0;
    if (M < 11 || M > 13) return fail(SIM_EINVAL, "sim_batch_create: tile_qubits must be 0 or 11..13");
    if (want_per_sm < 0) return fail(SIM_EINVAL, "sim_batch_create: ctas_per_sm must be >= 0");
    for (int c = 0; c < count; ++c) {
        if (n_qubits[c] < 1 || n_qubits[c] > 24) return fail(SIM_EINVAL, "sim_batch_create: qubit counts must be 1..24");
        if (gate_offsets[c + 1] < gate_offsets[c]) return fail(SIM_EINVAL, "sim_batch_create: offsets must not decrease");
        for (int64_t k = gate_offsets[c]; k < gate_offsets[c + 1]; ++k) {
            std::string why;
            if (validate_gate(n_qubits[c], gates[k], &why))
                return fail(SIM_EINVAL, "sim_batch_create: circuit " + std::to_string(c) + ": " + why);
        }
    }
    // host-side fault injection for tests: one circuit's pass waits for a tile that never comes
    const bool inject_stall = getenv("QSIM_INJECT_BATCH_STALL") != nullptr;

    std::vector<BCirc> circs(count);
    std::vector<BPass> passes;
    std::vector<StOp<float>> ops;
    int64_t state_amps = 0, parts = 0;
    double alg_flops = 0, alg_scratch = 0;
    for (int c = 0; c < count; ++c) {
        const int n = n_qubits[c];
        std::vector<SGate> g;
        lower_gates(gates + gate_offsets[c], (size_t)(gate_offsets[c + 1] - gate_offsets[c]), &g);
        for (const SGate &sg : g) alg_flops += sgate_flops(sg, n);
        merge_single_qubit(&g);
        const int nplan = std::max(n, M);           // below M qubits: phantom qubits that stay |0>
        std::vector<Pass> ps = form_passes(g, nplan, M);
        if (ps.empty()) {
            Pass empty_pass;
            for (int q = kLow; q < M; ++q) empty_pass.high.push_back(q);
            ps.push_back(empty_pass);
        }
        // scratch traffic the plan must make: every pass but the first reads
        // the state, every pass but the last writes it (8 B per amplitude)
        if (ps.size() > 1) alg_scratch += 2.0 * (double)(ps.size() - 1) * std::ldexp(8.0, nplan);
        PlanBuilder<float> pb{nplan, M, M - kThrBits, 2, {}, {}, 0};
        pb.allow_ramps = false;   // the batched kernel runs the tile engine without ramps
        BCirc bc{};
        bc.n = n;
        bc.npass = (int)ps.size();
        bc.ntiles = 1 << (nplan - M);
        bc.pass0 = (int64_t)passes.size();
        bc.part0 = parts;
        bc.state0 = 0;
        if (bc.ntiles > 1 || bc.npass > 1) {
            bc.state0 = state_amps;
            state_amps += (int64_t)1 << nplan;
        }
        parts += bc.ntiles;
        for (const Pass &p : ps) {
            BPass bp;
            memset(&bp, 0, sizeof bp);
            bp.op0 = (int64_t)(ops.size() + pb.ops.size());
            bp.nops = pb.schedule(p, g);
            bp.need = bc.ntiles;
            uint64_t q = (1ull << kLow) - 1ull;
            for (size_t i = 0; i < p.high.size(); ++i) {
                bp.geo.hpos[i] = p.high[i];
                q |= 1ull << p.high[i];
            }
            for (int b2 = 0; b2 < nplan; ++b2)
                if (!((q >> b2) & 1)) bp.geo.outer_pos[bp.geo.n_outer++] = b2;
            passes.push_back(bp);
        }
        if (inject_stall && c == 0 && bc.npass > 1) passes[bc.pass0 + 1].need = bc.ntiles + 1;
        ops.insert(ops.end(), pb.ops.begin(), pb.ops.end());
        circs[c] = bc;
    }
    // queue: pass index major, circuits by descending work, tiles ascending
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (int64_t)circs[a].ntiles * circs[a].npass > (int64_t)circs[b].ntiles * circs[b].npass;
    });
    int maxp = 0;
    for (const BCirc &c : circs) maxp = std::max(maxp, c.npass);
    std::vector<BItem> items;
    for (int p = 0; p < maxp; ++p)
        for (int c : order)
            if (p < circs[c].npass)
                for (int t = 0; t < circs[c].ntiles; ++t) items.push_back(BItem{c, p, t, 0});

    qsim_batch *b = new qsim_batch();
    b->count = count;
    b->tile_qubits = M;
    b->alg_flops = alg_flops;
    b->alg_scratch_bytes = alg_scratch;
    b->nitems = (int64_t)items.size();
    b->npasses = (int64_t)passes.size();
    b->nops = (int64_t)ops.size();
    int rc = SIM_OK;
    do {
        if (stream) {
            b->stream = (cudaStream_t)stream;
        } else {
            if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "batch stream");
                break;
            }
            b->owns_stream = true;
        }
        auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
        size_t off = 0;
        const size_t o_c = off; off += al(sizeof(BCirc) * count);
        const size_t o_p = off; off += al(sizeof(BPass) * passes.size());
        const size_t o_o = off; off += al(sizeof(StOp<float>) * std::max<size_t>(ops.size(), 1));
        const size_t o_i = off; off += al(sizeof(BItem) * items.size());
        const size_t o_ctl = off; off += al(sizeof(BCtl));
        const size_t o_d = off; off += al(sizeof(int) * passes.size());
        const size_t o_f = off; off += al(sizeof(int) * count);
        const size_t o_pa = off; off += al(sizeof(double) * parts);
        const size_t o_out = off; off += al(sizeof(double) * count);
        const size_t o_s = off; off += al(sizeof(float2) * std::max<int64_t>(state_amps, 1));
        b->scratch_bytes = off;
        if (cudaMalloc(&b->dev, off) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(SIM_ENOMEM, "sim_batch_create: device allocation failed");
            break;
        }
        char *d = (char *)b->dev;
        b->circs = (BCirc *)(d + o_c);
        b->passes = (BPass *)(d + o_p);
        b->ops = (StOp<float> *)(d + o_o);
        b->items = (BItem *)(d + o_i);
        b->ctl = (BCtl *)(d + o_ctl);
        b->done = (int *)(d + o_d);
        b->finished = (int *)(d + o_f);
        b->partial = (double *)(d + o_pa);
        b->out = (double *)(d + o_out);
        b->scratch = (float2 *)(d + o_s);
        if (cudaMemcpy(b->circs, circs.data(), sizeof(BCirc) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(b->passes, passes.data(), sizeof(BPass) * passes.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            (!ops.empty() && cudaMemcpy(b->ops, ops.data(), sizeof(StOp<float>) * ops.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
            cudaMemcpy(b->items, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "sim_batch_create: upload");
            break;
        }
        const void *kern = batch_kernel_for(M);
        const size_t smem = ((size_t)1 << M) * 2 * sizeof(float) + op_stage_bytes<float>();
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "batch smem attribute");
            break;
        }
        // up to two (13-qubit tiles) or three CTAs per SM
        if (cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "batch carveout attribute");
            break;
        }
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThr, smem) != cudaSuccess || per_sm < 1) {
            rc = fail(SIM_ECUDA, "sim_batch_create: persistent kernel does not fit on an SM");
            break;
        }
        if (want_per_sm > per_sm) {
            rc = fail(SIM_EINVAL, "sim_batch_create: ctas_per_sm " + std::to_string(want_per_sm) + " above the " +
                                      std::to_string(per_sm) + " that fit on an SM with " + std::to_string(M) +
                                      "-qubit tiles");
            break;
        }
        if (want_per_sm > 0) per_sm = want_per_sm;
        b->ctas_per_sm = per_sm;
        // persistent CTAs, at most one per resident slot.  A wait only ever
        // waits on items earlier in the queue (pass-major order), which CTAs
        // already running hold, so progress does not depend on residency.
        b->grid = sms * per_sm;
        // capture reset + persistent launch in a graph
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "capture stream");
            break;
        }
        cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        k_batch_reset<<<64, 256, 0, cs>>>(b->ctl, b->done, b->npasses, b->finished, count);
        if (M == 11)
            k_batch<11><<<b->grid, kThr, smem, cs>>>(b->scratch, b->circs, b->passes, b->ops, b->items, b->nitems,
                                                    b->ctl, b->done, b->finished, b->partial, b->out);
        else if (M == 12)
            k_batch<12><<<b->grid, kThr, smem, cs>>>(b->scratch, b->circs, b->passes, b->ops, b->items, b->nitems,
                                                    b->ctl, b->done, b->finished, b->partial, b->out);
        else
            k_batch<13><<<b->grid, kThr, smem, cs>>>(b->scratch, b->circs, b->passes, b->ops, b->items, b->nitems,
                                                    b->ctl, b->done, b->finished, b->partial, b->out);
        cudaError_t ce = cudaStreamEndCapture(cs, &b->graph);
        cudaStreamDestroy(cs);
        if (ce != cudaSuccess) {
            rc = cuda_fail(ce, "batch graph capture");
            break;
        }
        if ((ce = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) {
            rc = cuda_fail(ce, "batch graph instantiate");
            break;
        }
    } while (0);
    if (rc) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return SIM_OK;
}

extern "C" int sim_batch_create(int count, const int32_t *n_qubits, const int64_t *gate_offsets,
                                const sim_gate *gates, void *stream, qsim_batch **out)
{
    return sim_batch_create_opts(count, n_qubits, gate_offsets, gates, nullptr, stream, out);
}

extern "C" int sim_batch_config(qsim_batch *b, sim_batch_opts *used, double *alg_flops, double *alg_scratch_bytes)
{
    if (!b) return fail(SIM_EINVAL, "sim_batch_config: null batch");
    if (used) {
        memset(used, 0, sizeof *used);
        used->tile_qubits = b->tile_qubits;
        used->ctas_per_sm = b->ctas_per_sm;
    }
    if (alg_flops) *alg_flops = b->alg_flops;
    if (alg_scratch_bytes) *alg_scratch_bytes = b->alg_scratch_bytes;
    return SIM_OK;
}

extern "C" int sim_batch_run(qsim_batch *b, double *expz_out, int out_on_device)
{
    if (!b || !expz_out) return fail(SIM_EINVAL, "sim_batch_run: bad arguments");
    QSIM_CUDA(cudaGraphLaunch(b->exec, b->stream));
    QSIM_CUDA(cudaMemcpyAsync(expz_out, b->out, sizeof(double) * b->count,
                              out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    BCtl ctl;
    QSIM_CUDA(cudaMemcpyAsync(&ctl, b->ctl, sizeof ctl, cudaMemcpyDeviceToHost, b->stream));
    QSIM_CUDA(cudaStreamSynchronize(b->stream));
    if (ctl.status != 0) return fail(SIM_ETIMEOUT, "sim_batch_run: a dependency wait gave up");
    return SIM_OK;
}

extern "C" int sim_batch_info(qsim_batch *b, int64_t *items, int64_t *passes, int64_t *ops, int64_t *scratch_bytes,
                              int *grid)
{
    if (!b) return fail(SIM_EINVAL, "sim_batch_info: null batch");
    if (items) *items = b->nitems;
    if (passes) *passes = b->npasses;
    if (ops) *ops = b->nops;
    if (scratch_bytes) *scratch_bytes = (int64_t)b->scratch_bytes;
    if (grid) *grid = b->grid;
    return SIM_OK;
}

extern "C" int sim_batch_destroy(qsim_batch *b)
{
    batch_free(b);
    return SIM_OK;
}
