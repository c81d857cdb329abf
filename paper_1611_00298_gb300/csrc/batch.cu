// Batched solves: many independent systems of Eq. (8) (or D_DWF systems),
// possibly on several lattices, iterated together.  The heatbath needs 2 N_p
// such solves and the force 2 (Sec. 3.2, 3.3, 5.2); on small lattices each
// alone leaves most of the GPU idle and is bound by launch latency.
//
// Every system keeps its own reduction scratch and device scalars, so the
// iterations of all active systems can run concurrently: a chunk of 16 CG
// iterations of every active system is captured once into a CUDA graph
// (one stream per system, forked from and joined to an origin stream) and
// replayed; between replays the host reads each system's residual, does
// reliable updates and retires converged systems (which triggers a
// re-capture for the smaller active set).
#include "solver.h"

#include <chrono>
#include <memory>

#define BATCH_CHUNK 16

extern "C" int eofa_solve_batched(eofa_ctx* const* ctxs, int n, const eofa_solve_params* params,
                                  const double* const* b, double* const* x, eofa_solve_info* info) {
    if (!ctxs || n < 0 || !params || !b || !x) return EOFA_EINVAL;
    if (n == 0) return EOFA_OK;
    for (int i = 0; i < n; i++)
        if (!ctxs[i] || !b[i] || !x[i]) return EOFA_EINVAL;
    auto t0 = std::chrono::steady_clock::now();
    eofa_ctx* errctx = ctxs[0];
    std::vector<cudaStream_t> streams(n, nullptr);
    cudaStream_t origin = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> evs;
    std::vector<bool> prof_saved(n, false);
    double* rr_host = nullptr;
    int rc = EOFA_OK;
    try {
        std::vector<Solve> sv(n);
        std::vector<double*> bdev(n), xdev(n);
        EOFA_CUDA(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
        EOFA_CUDA(cudaMallocHost((void**)&rr_host, n * sizeof(double)));
        for (int i = 0; i < n; i++) {
            errctx = ctxs[i];
            EOFA_CUDA(cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking));
            size_t bytes = (size_t)ctxs[i]->V * ctxs[i]->Ls * 12 * 16;
            std::string tg = "_b" + std::to_string(i);
            bdev[i] = (double*)ctx_buffer(ctxs[i], "bt_b" + tg, bytes);
            xdev[i] = (double*)ctx_buffer(ctxs[i], "bt_x" + tg, bytes);
            double* red = (double*)ctx_buffer(ctxs[i], "bt_red" + tg, red_scratch_bytes());
            EOFA_CUDA(cudaMemsetAsync(red, 0, red_scratch_bytes(), streams[i]));
            EOFA_CUDA(cudaMemcpyAsync(bdev[i], b[i], bytes, cudaMemcpyHostToDevice, streams[i]));
            if (params[i].use_x0) EOFA_CUDA(cudaMemcpyAsync(xdev[i], x[i], bytes, cudaMemcpyHostToDevice, streams[i]));
            sv[i].setup(ctxs[i], params[i], bdev[i], xdev[i], tg, red, BATCH_CHUNK, streams[i]);
            if (!sv[i].trivial) sv[i].start_cg(streams[i]);
        }
        // fork/join events, 2 per system
        evs.resize(2 * n + 1);
        for (auto& e : evs) EOFA_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        std::vector<int> active, captured;
        std::vector<bool> finished(n, false);
        for (;;) {
            active.clear();
            for (int i = 0; i < n; i++) {
                if (finished[i]) continue;
                if (sv[i].done || sv[i].inf.iters >= sv[i].P.maxiter) {
                    errctx = ctxs[i];
                    if (sv[i].finish(xdev[i], streams[i])) {
                        finished[i] = true;
                        continue;
                    }
                    if (!sv[i].start_cg(streams[i])) continue;  // converged on restart: finish next round
                }
                active.push_back(i);
            }
            if (active.empty()) {
                bool all = true;
                for (int i = 0; i < n; i++) all = all && finished[i];
                if (all) break;
                continue;
            }
            if (active != captured) {
                if (exec) EOFA_CUDA(cudaGraphExecDestroy(exec));
                if (graph) EOFA_CUDA(cudaGraphDestroy(graph));
                exec = nullptr;
                graph = nullptr;
                for (int i : active) EOFA_CUDA(cudaStreamSynchronize(streams[i]));
                for (int i : active)
                    if (ctxs[i]->prof) { prof_saved[i] = ctxs[i]->prof->on; ctxs[i]->prof->on = false; }
                EOFA_CUDA(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
                EOFA_CUDA(cudaEventRecord(evs[2 * n], origin));
                for (int i : active) {
                    EOFA_CUDA(cudaStreamWaitEvent(streams[i], evs[2 * n], 0));
                    sv[i].enqueue(BATCH_CHUNK, streams[i]);
                    EOFA_CUDA(cudaEventRecord(evs[2 * i], streams[i]));
                    EOFA_CUDA(cudaStreamWaitEvent(origin, evs[2 * i], 0));
                }
                EOFA_CUDA(cudaStreamEndCapture(origin, &graph));
                for (int i : active)
                    if (ctxs[i]->prof) ctxs[i]->prof->on = prof_saved[i];
                EOFA_CUDA(cudaGraphInstantiate(&exec, graph, 0));
                captured = active;
                // the capture advanced the counters by one chunk; the first launch runs that chunk
            } else {
                for (int i : active) {
                    sv[i].it += BATCH_CHUNK;
                    sv[i].inf.iters += BATCH_CHUNK;
                }
            }
            // the graph runs on origin: order it after the host-side work queued on
            // each system's stream (restarts, reliable updates)
            for (int i : active) {
                EOFA_CUDA(cudaEventRecord(evs[2 * i + 1], streams[i]));
                EOFA_CUDA(cudaStreamWaitEvent(origin, evs[2 * i + 1], 0));
            }
            EOFA_CUDA(cudaGraphLaunch(exec, origin));
            EOFA_CUDA(cudaStreamSynchronize(origin));
            // each system's iteration counter stays a multiple of the chunk, so the
            // parities and residual-ring slots baked into the graph stay valid;
            // all residuals come back in one round trip
            for (size_t a = 0; a < active.size(); a++)
                EOFA_CUDA(cudaMemcpyAsync(rr_host + a, sv[active[a]].last_rr(), sizeof(double),
                                          cudaMemcpyDeviceToHost, origin));
            EOFA_CUDA(cudaStreamSynchronize(origin));
            for (size_t a = 0; a < active.size(); a++) {
                int i = active[a];
                errctx = ctxs[i];
                sv[i].check_value(rr_host[a], streams[i]);
            }
        }
        for (int i = 0; i < n; i++) {
            size_t bytes = (size_t)ctxs[i]->V * ctxs[i]->Ls * 12 * 16;
            EOFA_CUDA(cudaMemcpyAsync(x[i], xdev[i], bytes, cudaMemcpyDeviceToHost, streams[i]));
            EOFA_CUDA(cudaStreamSynchronize(streams[i]));
            eofa_solve_info inf = sv[i].inf;
            inf.true_resid = sv[i].true_rel;
            inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            inf.status = !std::isfinite(sv[i].true_rel) ? EOFA_ENUMERIC
                                                         : (sv[i].true_rel > sv[i].P.tol ? EOFA_ENOTCONV : EOFA_OK);
            if (info) info[i] = inf;
            if (inf.status != EOFA_OK && rc == EOFA_OK) {
                rc = inf.status;
                ctxs[i]->err = "batched solve " + std::to_string(i) + " did not converge";
            }
        }
    } catch (const eofa_error& e) {
        cudaStreamCaptureStatus cs;
        if (origin && cudaStreamIsCapturing(origin, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(origin, &g);
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
        rc = fail(errctx, e.code, e.msg);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto& e : evs) cudaEventDestroy(e);
    for (auto& s : streams)
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    if (origin) cudaStreamDestroy(origin);
    if (rr_host) cudaFreeHost(rr_host);
    return rc;
}
