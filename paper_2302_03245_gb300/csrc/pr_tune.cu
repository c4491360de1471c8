// pr_tune.cu -- launch parameters of a graph (pull bins, block budget, push/pull
// switch) and the autotuner that chooses them by timing trial rounds.
//
// A trial is an ordinary solve through pr_solve_ex with host-driven rounds and
// the per-kernel CUDA-event profile: the dense gather trial runs IFP2 in PULL
// mode with a threshold below every residual (every non-dangling row active)
// for a few rounds; the push trial runs IFP2 in PUSH mode.  Nothing here adds
// arithmetic of its own: the tuner only reads timings.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pr_internal.cuh"

using namespace pr;

namespace {

void fill_tuning(const pr_graph *g, pr_tuning *t) {
    std::memset(t, 0, sizeof(*t));
    for (int k = 0; k < kNumThr; k++) t->pull_thr[k] = g->thr[k];
    t->block_budget = g->block_budget;
    t->pull_ratio = g->pull_ratio;
    // rows per bin of the non-dangling rows: each referenced range (the class,
    // or each of its levels) is split at its 6 bounds; the unreferenced rows
    // (no in-edges) run one lane each
    for (int k = 0; k < g->nranges - 1; k++) {
        int32_t a = g->range_lo[k];
        for (int t2 = 0; t2 < kNumThr; t2++) {
            const int32_t b = g->bounds[k * kNumThr + t2];
            t->bin_rows[t2] += b - a;
            a = b;
        }
        t->bin_rows[kNumThr] += g->range_hi[k] - a;
    }
    t->bin_rows[kNumThr] += g->G.n_nd - g->G.n_ref;
    t->pull_blocks = g->plan_nd.nblocks;  // the plan of a double-float or FP32 solve
}

struct Trial {
    pr_graph *g;
    pr_prec prec;
    double *dout;
    double spent_ms = 0.0;
    int32_t n_nd;

    // mean duration of a dense gather launch (ms), over `rounds` rounds
    pr_status pull_round(int rounds, double *ms) {
        pr_kernel_profile prof;
        pr_opts o{};
        o.mode = PR_MODE_PULL;
        o.max_rounds = rounds;
        o.use_graph = -1;
        o.xi_act = 1e-300;
        o.profile = &prof;
        pr_stats st;
        const pr_status s = pr_solve_ex(g, 0.85, 1e-300, PR_IFP2, prec, nullptr, &o, dout, 1, &st);
        if (s != PR_OK && s != PR_ENOTCONV) return s;
        double all = 0;
        for (int k = 0; k < PR_K_KINDS; k++) all += prof.ms[k];
        spent_ms += all;
        *ms = prof.launches[PR_K_PULL] ? prof.ms[PR_K_PULL] / prof.launches[PR_K_PULL] : 0.0;
        return PR_OK;
    }

    // push rounds: device ms per pushed edge and per activation scan
    pr_status push_rounds(int rounds, double *ms_per_edge, double *act_ms) {
        pr_kernel_profile prof;
        std::vector<int64_t> E(rounds + 2, 0), F(rounds + 2, 0);
        std::vector<double> R(rounds + 2, 0.0);
        std::vector<int8_t> M(rounds + 2, 0);
        pr_opts o{};
        o.mode = PR_MODE_PUSH;
        o.max_rounds = rounds;
        o.use_graph = -1;
        o.profile = &prof;
        o.trace_cap = rounds + 2;
        o.trace_E = E.data();
        o.trace_F = F.data();
        o.trace_R = R.data();
        o.trace_mode = M.data();
        pr_stats st;
        // a PPR-like start (one seed at the first referenced row, the highest
        // in-degree) grows the frontier from one vertex: the trial sees push
        // rounds of many sizes
        int32_t seed = 0;  // caller id of internal row 0
        PR_CK(cudaMemcpyAsync(&seed, g->G.perm, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
        PR_CK(cudaStreamSynchronize(g->stream));
        const double one = 1.0;
        pr_pvec p{1, &seed, &one, 0};
        const pr_status s = pr_solve_ex(g, 0.85, 1e-300, PR_IFP2, prec, &p, &o, dout, 1, &st);
        if (s != PR_OK && s != PR_ENOTCONV) return s;
        double all = 0;
        for (int k = 0; k < PR_K_KINDS; k++) all += prof.ms[k];
        spent_ms += all;
        long long edges = 0;
        for (int t = 0; t < std::min<int>(st.rounds, rounds + 2); t++)
            if (M[t] == 1) edges += E[t];
        *ms_per_edge = edges > 0 ? prof.ms[PR_K_PUSH] / (double)edges : 0.0;
        *act_ms = prof.launches[PR_K_ACTIVATE] ? prof.ms[PR_K_ACTIVATE] / prof.launches[PR_K_ACTIVATE] : 0.0;
        return PR_OK;
    }
};

void append(std::string &rep, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
void append(std::string &rep, const char *fmt, ...) {
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    rep += buf;
}

}  // namespace

extern "C" pr_status pr_graph_get_tuning(const pr_graph *g, pr_tuning *t) {
    if (!g || !t) return fail(PR_EINVAL, "pr_graph_get_tuning: NULL argument");
    fill_tuning(g, t);
    return PR_OK;
}

extern "C" pr_status pr_graph_set_tuning(pr_graph *g, const pr_tuning *t) {
    if (!g || !t) return fail(PR_EINVAL, "pr_graph_set_tuning: NULL argument");
    if (!(t->pull_ratio >= 0.0) || !std::isfinite(t->pull_ratio))
        return fail(PR_EINVAL, "pull_ratio must be finite and >= 0");
    PR_TRY(set_bins(g, t->pull_thr, t->block_budget, g->stream));
    if (t->pull_ratio > 0) g->pull_ratio = t->pull_ratio;
    return PR_OK;
}

extern "C" pr_status pr_graph_autotune(pr_graph *g, pr_prec prec, double max_ms, pr_tuning *out, char *report,
                                       size_t report_len) {
    if (!g) return fail(PR_EINVAL, "pr_graph_autotune: NULL graph");
    if (prec != PR_FP64 && prec != PR_FP32 && prec != PR_DF64) return fail(PR_EINVAL, "unknown precision");
    if (!(max_ms >= 0.0) || !std::isfinite(max_ms)) return fail(PR_EINVAL, "max_ms must be finite and >= 0");
    if (max_ms == 0.0) max_ms = 3000.0;
    std::string rep;
    if (g->G.n_nd == 0 || g->G.m == 0) {  // nothing to gather or push
        if (out) fill_tuning(g, out);
        return PR_OK;
    }
    Buf dout;
    PR_TRY(dout.alloc(sizeof(double) * g->G.n, g->stream));
    Trial T{g, prec, dout.as<double>(), 0.0, g->G.n_nd};
    const int sms = std::max(g->num_sms, 1);
    int32_t cur_thr[kNumThr];
    for (int k = 0; k < kNumThr; k++) cur_thr[k] = g->thr[k];
    const int32_t cur_budget = g->block_budget;
    constexpr int kRounds = 5;  // round 0 activates; rounds 1..4 are dense gathers

    // warm-up (workspace allocation, first-touch) and the current tuning's time
    double ms = 0.0, best_ms = 0.0;
    PR_TRY(T.pull_round(kRounds, &ms));
    PR_TRY(T.pull_round(kRounds, &best_ms));
    int32_t best_thr[kNumThr];
    for (int k = 0; k < kNumThr; k++) best_thr[k] = cur_thr[k];
    int32_t best_budget = cur_budget;
    append(rep, "current thr=[%d,%d,%d,%d,%d,%d] budget=%d: %.4f ms/round\n", cur_thr[0], cur_thr[1], cur_thr[2],
           cur_thr[3], cur_thr[4], cur_thr[5], cur_budget, best_ms);
    // candidates: the block-row threshold, the warp-row threshold (the finer
    // lane bins halve below it), the block budget in blocks per SM
    const int32_t t0s[] = {1024, 4096, 16384};
    const int32_t t1s[] = {16, 32, 64};
    const int bpsm[] = {8, 16, 32};
    bool out_of_time = false;
    for (int32_t t1 : t1s) {
        for (int32_t t0 : t0s) {
            for (int b : bpsm) {
                if (T.spent_ms > max_ms) {
                    out_of_time = true;
                    break;
                }
                int32_t thr[kNumThr] = {t0, t1, std::max(t1 / 2, 1), std::max(t1 / 4, 1), std::max(t1 / 8, 1),
                                        std::max(t1 / 16, 1)};
                const int32_t budget = std::min(sms * b, kMaxBlocks / 2);
                if (set_bins(g, thr, budget, g->stream) != PR_OK) continue;
                double m1 = 0, m2 = 0;
                PR_TRY(T.pull_round(kRounds, &m1));
                PR_TRY(T.pull_round(kRounds, &m2));
                const double m = std::min(m1, m2);
                append(rep, "thr=[%d,%d,%d,%d,%d,%d] budget=%d: %.4f ms/round\n", thr[0], thr[1], thr[2], thr[3],
                       thr[4], thr[5], budget, m);
                if (m < best_ms) {
                    best_ms = m;
                    for (int k = 0; k < kNumThr; k++) best_thr[k] = thr[k];
                    best_budget = budget;
                }
            }
            if (out_of_time) break;
        }
        if (out_of_time) break;
    }
    PR_TRY(set_bins(g, best_thr, best_budget, g->stream));
    // push/pull switch: a push round costs about act + b * E (E = edges pushed);
    // a pull round costs best_ms.  Pull from E* = (best_ms - act) / b on.
    if (!out_of_time || T.spent_ms < 2.0 * max_ms) {
        double b = 0.0, act = 0.0;
        PR_TRY(T.push_rounds(12, &b, &act));
        const int64_t m_valid = std::max<int64_t>(g->G.m - g->info.m_d, 1);
        if (b > 0.0) {
            const double e_star = std::max(best_ms - act, 0.0) / b;
            const double ratio = std::min(std::max(e_star / (double)m_valid, 0.002), 1.0);
            g->pull_ratio = ratio;
            append(rep, "push: %.3e ms/edge, activation %.4f ms; pull %.4f ms -> switch at %.0f edges (ratio %.4f)\n",
                   b, act, best_ms, e_star, ratio);
        }
    }
    append(rep, "chosen thr=[%d,%d,%d,%d,%d,%d] budget=%d pull_ratio=%.4f; trial device time %.1f ms%s\n",
           best_thr[0], best_thr[1], best_thr[2], best_thr[3], best_thr[4], best_thr[5], best_budget, g->pull_ratio,
           T.spent_ms, out_of_time ? " (time bound reached)" : "");
    if (report && report_len) {
        const size_t k = std::min(report_len - 1, rep.size());
        std::memcpy(report, rep.data(), k);
        report[k] = '\0';
    }
    if (out) fill_tuning(g, out);
    return PR_OK;
}
