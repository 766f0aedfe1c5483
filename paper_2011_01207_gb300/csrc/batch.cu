// Batched replicas: many independent systems of uneven size advanced by one CUDA-graph
// launch. Each replica is an ordinary context on its own stream; one step of every
// replica (permanent field, optional learned guess, the PCG solve with its conditional
// WHILE loop, energy and forces) is captured as a parallel branch of a single graph, so a
// batch step is one graph launch and the replicas' kernels fill the GPU together.
// The paper runs many independent trajectories as separate jobs (adaptive sampling,
// Sec. 3 perspectives); on one GB300 they share the device instead.
//
// ap_autotune() picks launch shapes per context by timing the candidates.
#include "common.cuh"

#include <algorithm>
#include <vector>

int ap_learned_guess(ap_ctx *ctx, const void *d_packed, double *d_mu0);
int hist_guess_launch(ap_ctx *ctx, const double *g, const double *h, double *out, cudaStream_t s);
int hist_push_launch(ap_ctx *ctx, const double *g, const double *mu, double *h, cudaStream_t s);
int hist_adaptive_launch(ap_ctx *ctx, const double *g, double *h, double *out, cudaStream_t s);
int hist_push3_launch(ap_ctx *ctx, const double *g, const double *mu, double *h, cudaStream_t s);
int pme_stage_launch(ap_ctx *ctx, int stage, cudaStream_t s);
int dipole_operator_into(ap_ctx *ctx, cudaStream_t main, cudaStream_t aux);

struct ap_batch {
    std::vector<ap_ctx *> ctxs;
    cudaStream_t bs = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int capture_one(ap_ctx *c, const ap_batch_step &st) {
    int r = permanent_field(c, st.d_xyz, st.d_mpole, st.d_frame, st.d_alpha, nullptr);
    if (r) return r;
    const double *guess = nullptr;
    if ((st.d_hist || st.d_hist_lsq) && !st.d_mlp_packed)
        return ap_fail(c, AP_ERR_ARG, "the trajectory guess needs the learned guess");
    if (st.d_mlp_packed) {
        if (!st.d_mu0) return ap_fail(c, AP_ERR_ARG, "learned guess needs d_mu0 scratch");
        if ((r = ap_learned_guess(c, st.d_mlp_packed, st.d_mu0))) return r;
        guess = st.d_mu0;
    }
    double *hist_out = st.d_hist ? st.d_hist + 12L * c->n : nullptr;   // slot 5 of [5][n][3]
    if (st.d_hist_lsq) {
        double *out = st.d_hist_lsq + 18L * c->n;                        // the guess, after six vectors
        if ((r = hist_adaptive_launch(c, st.d_mu0, st.d_hist_lsq, out, c->s0))) return ap_fail(c, r, "history guess");
        guess = out;
    } else if (st.d_hist) {
        if ((r = hist_guess_launch(c, st.d_mu0, st.d_hist, hist_out, c->s0))) return ap_fail(c, r, "history guess");
        guess = hist_out;
    }
    if ((r = induced_dipoles_pcg(c, guess, st.tol_debye, st.max_iter, st.d_mu, nullptr)) < 0) return r;
    if (st.d_hist_lsq) {
        if ((r = hist_push3_launch(c, st.d_mu0, st.d_mu, st.d_hist_lsq, c->s0))) return ap_fail(c, r, "history push");
    } else if (st.d_hist) {
        if ((r = hist_push_launch(c, st.d_mu0, st.d_mu, st.d_hist, c->s0))) return ap_fail(c, r, "history push");
    }
    if (st.d_energy && st.d_forces)
        if ((r = polarization_energy_forces(c, st.d_mu, st.d_energy, st.d_forces, st.d_virial))) return r;
    return AP_OK;
}

}  // namespace

extern "C" {

int ap_batch_create(ap_batch **out, ap_ctx *const *ctxs, int n) {
    if (!out || !ctxs || n <= 0) return ap_fail(nullptr, AP_ERR_ARG, "bad batch arguments");
    *out = nullptr;
    ap_batch *b = new ap_batch();
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !ctxs[i]->s0) {
            delete b;
            return ap_fail(nullptr, AP_ERR_ARG, "every replica needs its own non-default stream");
        }
        b->ctxs.push_back(ctxs[i]);
    }
    if (cudaStreamCreateWithFlags(&b->bs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        delete b;
        return ap_fail(nullptr, AP_ERR_CUDA, "batch stream/event");
    }
    b->join.resize(n);
    for (int i = 0; i < n; ++i) cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    *out = b;
    return AP_OK;
}

int ap_batch_capture(ap_batch *b, const ap_batch_step *steps) {
    if (!b || !steps) return ap_fail(nullptr, AP_ERR_ARG, "null batch");
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    // a new capture starts a new trajectory for the history guesses
    for (ap_ctx *c : b->ctxs)
        if (cudaMemset(c->hist_count, 0, sizeof(int)) != cudaSuccess)
            return ap_fail(nullptr, AP_ERR_CUDA, "history counter reset");
    cudaError_t e = cudaStreamBeginCapture(b->bs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    cudaEventRecord(b->fork, b->bs);
    int rc = AP_OK;
    for (size_t i = 0; i < b->ctxs.size() && rc == AP_OK; ++i) {
        ap_ctx *c = b->ctxs[i];
        cudaStreamWaitEvent(c->s0, b->fork, 0);
        rc = capture_one(c, steps[i]);
        cudaEventRecord(b->join[i], c->s0);
        cudaStreamWaitEvent(b->bs, b->join[i], 0);
        if (rc) ap_fail(nullptr, rc, "replica " + std::to_string(i) + ": " + c->err);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->bs, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->exec, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    return AP_OK;
}

int ap_batch_launch(ap_batch *b, void *stream) {
    if (!b || !b->exec) return ap_fail(nullptr, AP_ERR_STATE, "ap_batch_capture() must come first");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    return AP_OK;
}

void ap_batch_destroy(ap_batch *b) {
    if (!b) return;
    if (b->bs) cudaStreamSynchronize(b->bs);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->fork) cudaEventDestroy(b->fork);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->bs) cudaStreamDestroy(b->bs);
    delete b;
}

int ap_autotune(ap_ctx *ctx, int reps, int *h_choice) {
    if (!ctx || reps < 1) return AP_ERR_ARG;
    ctx->err.clear();
    if (!ctx->config_valid) return ap_fail(ctx, AP_ERR_STATE, "permanent_field() must come first");
    cudaEvent_t a, z;
    AP_CUDA(cudaEventCreate(&a));
    AP_CUDA(cudaEventCreate(&z));
    auto time_it = [&](auto launch) -> float {
        float best = 1e30f;
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(a, ctx->s0);
            launch();
            cudaEventRecord(z, ctx->s0);
            cudaEventSynchronize(z);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, z);
            best = ms < best ? ms : best;
        }
        return best;
    };
    // whole PCG solves (four iterations from alpha E, as one graph launch each) for every
    // combination of the real-space matvec's CTAs per SM (as many as fit, r, then r - 1,
    // r - 2, r - 3, r - 4, r - 6 and 3, those from 3 to r - 1) and the PME spread/gather
    // block size (64, 128 and 256 threads): what counts is the matvec running concurrently
    // with the reciprocal branch inside the solve, and the matvec's grid decides how much
    // room the PME kernels find on the SMs (a resident grid fills every SM's registers)
    auto forget = [&] {
        if (ctx->solve_exec) cudaGraphExecDestroy(ctx->solve_exec);
        ctx->solve_exec = nullptr;
        ctx->graph_ok = 0;
        ctx->graph_tried = 0;
    };
    const int r = real_matvec_resident_per_sm(ctx);
    std::vector<int> per_sm = {0};
    for (int d : {r - 1, r - 2, r - 3, r - 4, r - 6, 3})
        if (d >= 3 && d < r && std::find(per_sm.begin(), per_sm.end(), d) == per_sm.end()) per_sm.push_back(d);
    const int thr[3] = {64, 128, 256};
    float best = 1e30f;
    int best_per_sm = 0, best_thr = 128;
    for (int d : per_sm)
        for (int th : thr) {
            ctx->tune_mv_per_sm = d;
            ctx->tune_pme_threads = th;
            forget();
            int rc = pcg_solve(ctx, nullptr, 1e-300, 4, ctx->frc, nullptr);   // captures the loop
            if (rc < 0) return rc;
            float t = time_it([&] { pcg_solve(ctx, nullptr, 1e-300, 4, ctx->frc, nullptr); });
            if (t < best) { best = t; best_per_sm = d; best_thr = th; }
        }
    ctx->tune_mv_per_sm = best_per_sm;
    ctx->tune_pme_threads = best_thr;
    // the solve graphs captured the old launch shapes: capture again at the next solve
    forget();
    if (ctx->diis_exec) cudaGraphExecDestroy(ctx->diis_exec);
    ctx->diis_exec = nullptr;
    dp_forget_graph(ctx);
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    AP_CUDA(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * 3 * ctx->n_pad, ctx->s0));
    AP_CUDA(cudaMemsetAsync(ctx->frc, 0, sizeof(double) * 3 * ctx->n_pad, ctx->s0));
    AP_CUDA(cudaStreamSynchronize(ctx->s0));
    AP_CUDA(cudaGetLastError());
    if (h_choice) {
        h_choice[0] = best_per_sm;
        h_choice[1] = best_thr;
    }
    return AP_OK;
}

}  // extern "C"
