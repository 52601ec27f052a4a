// learned.cu -- SIM_PLAN_LEARNED: the circuit is cut into windows of
// consecutive gates; for every window and every feasible plan variant the
// host computes a feature row (rows in parallel on the host cores), the cost
// model (mlp.cu) predicts the log run time of all rows in one batched forward
// pass on the GPU, and the cheaper of two plans runs: each window with its
// own cheapest variant, or the whole circuit with the one variant whose
// windows sum to the least (one variant over many windows lets the block and
// pass planners work across window boundaries, which per-window predictions
// cannot see, so a mix must win by a margin).  Without a model the greedy
// fixed-k plan runs (fused blocks of the largest k whose tile fits): it is
// both the fallback and the yardstick the learned plans are measured against.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "internal.cuh"

extern "C" int sim_mlp_forward(qsim_mlp *m, const float *x, int64_t rows, float *y, int on_device);

namespace qsim {

namespace {

struct Window {
    size_t first, count;
};

int variant_opts(int v, sim_plan_opts *o)
{
    memset(o, 0, sizeof *o);
    if (v == 0) { o->plan = SIM_PLAN_PER_GATE; return 0; }
    if (v == 1 || v == 2) { o->plan = SIM_PLAN_STAGED; o->tile_qubits = (v == 1) ? 12 : 13; return 0; }
    if (v >= 3 && v <= 6) { o->plan = SIM_PLAN_FUSED; o->fuse_k = v; return 0; }
    return -1;
}

bool feasible(int n, int dtype, int v)
{
    if (v == 0) return true;
    if (v == 1) return n >= 12 && dtype == SIM_C64 ? true : (v == 1 && n >= 12 && dtype == SIM_C128);
    if (v == 2) return n >= 13 && dtype == SIM_C64;
    return dtype == SIM_C64 && n >= v + 7;
}

}  // namespace

int plan_features(int n, int dtype, const sim_gate *gates, size_t n_gates, int v, float *out)
{
    if (!feasible(n, dtype, v)) return SIM_EUNSUPPORTED;
    std::vector<SGate> g;
    lower_gates(gates, n_gates, &g);
    double dense = 0, ctrlx = 0, diag = 0;
    uint64_t touched = 0;
    for (const SGate &s : g) {
        touched |= s.xq() | s.dq();
        if (s.xq()) (s.ctrl ? ctrlx : dense) += 1;
        else diag += 1;
    }
    const double m = (double)g.size();
    double launches = m, ops = 0, lc = 0;
    if (v == 1 || v == 2) {
        int64_t p = 0, o = 0, l = 0;
        if (describe_staged(n, dtype, gates, n_gates, v == 1 ? 12 : 13, &p, &o, &l, nullptr, 0, nullptr)) return SIM_EINVAL;
        launches = (double)p;
        ops = (double)o;
        lc = (double)l;
    } else if (v >= 3) {
        int64_t b = 0;
        // block count from the one-qubit-at-a-time planner: cheap enough to
        // run for every window and variant; the run plans deeper, and the
        // model learns the mapping from these features to its timings
        describe_fused(n, gates, n_gates, v, &b, fused_feature_depth());
        launches = (double)b;
    }
    for (int i = 0; i < SIM_FEATURES; ++i) out[i] = 0.f;
    out[0] = (float)(n / 32.0);
    out[1] = (float)(std::log2(m + 1.0) / 12.0);
    out[2] = (float)(m > 0 ? dense / m : 0);
    out[3] = (float)(m > 0 ? diag / m : 0);
    out[4] = (float)(m > 0 ? ctrlx / m : 0);
    out[5] = (float)(__builtin_popcountll(touched) / (double)n);
    out[6 + v] = 1.f;
    out[13] = (float)(std::log2(launches + 1.0) / 12.0);
    out[14] = (float)(std::log2(ops + 1.0) / 14.0);
    out[15] = (float)(lc / (ops + 1.0));
    return SIM_OK;
}

// The learned plan's choice for a complex64 register with a cost model: one
// variant per window of max(64, 8n) gates (into *best, also kept as the
// handle's last plan).
int learned_choose(qsim_state *s, const sim_gate *gates, size_t n_gates, std::vector<int> *best_out)
{
    // windows of about eight layers of single-qubit gates
    const size_t W = (size_t)std::max(64, 8 * s->n);
    std::vector<Window> win;
    for (size_t f = 0; f < n_gates; f += W) win.push_back(Window{f, std::min(W, n_gates - f)});
    const size_t nw = win.size();
    // predicted log times of the feasible variants of some segments, the
    // feature rows in parallel on the host threads, one batched forward pass
    struct Pred { size_t seg; int v; float p; };
    auto predict = [&](const std::vector<Window> &segs, std::vector<Pred> *out) -> int {
        std::vector<std::pair<size_t, int>> cand;
        for (size_t w = 0; w < segs.size(); ++w)
            for (int v = 0; v < SIM_VARIANTS; ++v)
                if (feasible(s->n, s->dtype, v)) cand.push_back({w, v});
        std::vector<float> feat(cand.size() * SIM_FEATURES);
        std::vector<char> ok(cand.size(), 0);
        parallel_for(cand.size(), [&](size_t r) {
            const Window &w = segs[cand[r].first];
            ok[r] = plan_features(s->n, s->dtype, gates + w.first, w.count, cand[r].second,
                                  feat.data() + r * SIM_FEATURES) == SIM_OK;
        });
        std::vector<float> rows;
        out->clear();
        for (size_t r = 0; r < cand.size(); ++r)
            if (ok[r]) {
                rows.insert(rows.end(), feat.begin() + r * SIM_FEATURES, feat.begin() + (r + 1) * SIM_FEATURES);
                out->push_back(Pred{cand[r].first, cand[r].second, 0.f});
            }
        std::vector<float> pred(out->size());
        if (!out->empty())
            if (int rc = sim_mlp_forward((qsim_mlp *)s->cost_model, rows.data(), (int64_t)out->size(), pred.data(), 0))
                return rc;
        for (size_t r = 0; r < out->size(); ++r) (*out)[r].p = pred[r];
        return SIM_OK;
    };
    std::vector<Pred> pw;
    if (int rc = predict(win, &pw)) return rc;
    std::vector<int> &best = *best_out;
    best.assign(nw, -1);
    std::vector<float> bestp(nw, 0.f);
    for (const Pred &x : pw)
        if (best[x.seg] < 0 || x.p < bestp[x.seg]) { best[x.seg] = x.v; bestp[x.seg] = x.p; }
    bool agree = true;
    for (size_t w = 0; w < nw; ++w) agree = agree && best[w] >= 0 && best[w] == best[0];
    // When the windows disagree, the mix of per-window argmins is compared
    // with the best single variant for the whole circuit, whose time is
    // predicted as the sum of its window predictions (running it as one call
    // can only do better: its block and pass planners then work across window
    // boundaries; fused k = 5 on the 30-qubit workload took 356 ms as four
    // windows and 261 ms as one call).  The mix must win by a margin: each
    // prediction is off by about the model's log-time RMSE (0.06-0.08 on its
    // training timings), so the mix runs only if it is predicted faster by
    // twice that error, a factor exp(-2 x 0.084).  No planner runs over the
    // whole circuit here: those feature rows cost more host time than the
    // windows' rows together.
    if (!agree && nw > 1) {
        constexpr double kMixMargin = 0.845;
        std::vector<double> uni(SIM_VARIANTS, 0.0);
        std::vector<size_t> seen(SIM_VARIANTS, 0);
        for (const Pred &x : pw) {
            uni[x.v] += std::exp((double)x.p);
            seen[x.v]++;
        }
        int whole_v = -1;
        for (int v = 0; v < SIM_VARIANTS; ++v)
            if (seen[v] == nw && (whole_v < 0 || uni[v] < uni[whole_v])) whole_v = v;
        double mix = 0;
        bool all = true;
        for (size_t w = 0; w < nw; ++w) {
            if (best[w] < 0) all = false;
            else mix += std::exp((double)bestp[w]);
        }
        if (whole_v >= 0 && (!all || mix > kMixMargin * uni[whole_v])) std::fill(best.begin(), best.end(), whole_v);
    }
    s->last_plan.assign(best.begin(), best.end());
    return SIM_OK;
}

int apply_circuit_learned(qsim_state *s, const sim_gate *gates, size_t n_gates, const sim_plan_opts &o)
{
    if (!s->cost_model) {
        // the greedy fixed-k plan: the largest block size whose tile fits
        // (k = 6 from 13 qubits; complex128 k = 4 from 11), per gate below
        const int kmax = s->dtype == SIM_C128 ? 4 : 6;
        const int k = std::min(kmax, s->n - 7);
        if (k >= (s->dtype == SIM_C128 ? 4 : 3)) {
            s->last_plan.assign(1, k);
            sim_plan_opts fo{};
            fo.plan = SIM_PLAN_FUSED;
            fo.fuse_k = k;
            return apply_circuit_fused(s, gates, n_gates, fo);
        }
        s->last_plan.assign(1, 0);
        for (size_t i = 0; i < n_gates; ++i)
            if (int rc = launch_pair_gate(s, make_pair_gate(gates[i]))) return rc;
        return SIM_OK;
    }
    if (n_gates == 0) {
        s->last_plan.clear();
        return SIM_OK;
    }
    if (s->dtype == SIM_C128) {
        // complex128: the per-gate and register-tile kernels are bound by this
        // GPU's narrow FP64 pipe, while 4-qubit fused blocks run on the FP16
        // tensor cores as exact integer digit-plane products (fused64.cu).
        // Measured at 30 qubits (Haar layers + CZ, depth 20): fused 1276 ms
        // against 12837 ms per gate; 28-qubit QFT: 253 against 351 ms.  So the
        // fused plan runs wherever a 4-qubit block's tile fits (n >= 11), the
        // per-gate plan below that; the model (trained on complex64 timings)
        // is not consulted.
        if (s->n >= 11) {
            s->last_plan.assign(1, 4);
            sim_plan_opts fo{};
            fo.plan = SIM_PLAN_FUSED;
            fo.fuse_k = 4;
            return apply_circuit_fused(s, gates, n_gates, fo);
        }
        s->last_plan.assign(1, 0);
        for (size_t k = 0; k < n_gates; ++k)
            if (int rc = launch_pair_gate(s, make_pair_gate(gates[k]))) return rc;
        return SIM_OK;
    }
    std::vector<int> best;
    if (int rc = learned_choose(s, gates, n_gates, &best)) return rc;
    const size_t W = (size_t)std::max(64, 8 * s->n);
    std::vector<Window> win;
    for (size_t f = 0; f < n_gates; f += W) win.push_back(Window{f, std::min(W, n_gates - f)});
    // consecutive windows with the same variant run as one call, so the tile
    // and block planners see the whole run of gates
    for (size_t w = 0; w < win.size();) {
        size_t e = w + 1;
        while (e < win.size() && best[e] == best[w]) ++e;
        const size_t first = win[w].first, count = win[e - 1].first + win[e - 1].count - first;
        sim_plan_opts vo;
        variant_opts(best[w] < 0 ? 0 : best[w], &vo);
        int rc;
        if (vo.plan == SIM_PLAN_PER_GATE) {
            rc = SIM_OK;
            for (size_t k = 0; k < count && rc == SIM_OK; ++k) rc = launch_pair_gate(s, make_pair_gate(gates[first + k]));
        } else if (vo.plan == SIM_PLAN_STAGED) {
            rc = apply_circuit_staged(s, gates + first, count, vo);
        } else {
            rc = apply_circuit_fused(s, gates + first, count, vo);
        }
        if (rc) return rc;
        w = e;
    }
    return SIM_OK;
}

}  // namespace qsim

using namespace qsim;

extern "C" int sim_plan_features(int n, int dtype, const sim_gate *gates, size_t n_gates, int variant, float *out)
{
    set_error("");
    if (n < 1 || n > 34 || !out || variant < 0 || variant >= SIM_VARIANTS || (n_gates && !gates))
        return fail(SIM_EINVAL, "sim_plan_features: bad arguments");
    for (size_t k = 0; k < n_gates; ++k) {
        std::string why;
        if (validate_gate(n, gates[k], &why)) return fail(SIM_EINVAL, "sim_plan_features: " + why);
    }
    const int rc = plan_features(n, dtype, gates, n_gates, variant, out);
    if (rc == SIM_EUNSUPPORTED) return fail(rc, "sim_plan_features: variant not feasible for this register");
    return rc;
}

extern "C" int sim_set_cost_model(sim_t s, qsim_mlp *m)
{
    if (!s) return fail(SIM_EINVAL, "sim_set_cost_model: null handle");
    s->cost_model = m;
    return SIM_OK;
}

extern "C" int sim_last_plan(sim_t s, int32_t *variants, size_t cap, size_t *len)
{
    if (!s) return fail(SIM_EINVAL, "sim_last_plan: null handle");
    if (len) *len = s->last_plan.size();
    for (size_t i = 0; variants && i < cap && i < s->last_plan.size(); ++i) variants[i] = s->last_plan[i];
    return SIM_OK;
}
