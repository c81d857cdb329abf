// Batched solves: many independent systems of Eq. (8) (or D_DWF systems),
// possibly on several lattices.  The heatbath needs 2 N_p such solves and
// the force 2 (Sec. 3.2, 3.3, 5.2); the mass pairs of several EOFA factors
// add more.
//
// Systems on the same (small) lattice and with the same inner precision
// form a group (at most MR_MAX systems); a system on a large lattice is a
// group of its own (MR_SINGLE_SITES).  A group iterates its systems in lock
// step with the multi-system kernels of mrhs.cuh: the five-launch form of
// the CG iteration of solver.cu, each launch for all of them, each link row
// and neighbour index fetched once for the whole group.  The CG loop of a group runs on the device: a CUDA graph
// holds one WHILE conditional node whose body is K CG iterations of every
// active system followed by a one-block decision kernel; the kernel reads
// each system's |r|^2 and keeps the loop going until some system has
// reached its inner target, needs an FP64 reliable update, diverges or
// runs out of iterations.  Only then does the host look at the group: it
// does the reliable updates and the true-residual checks of solver.cu,
// retires converged systems (re-capturing the graph for the smaller set)
// and relaunches.  Lock-step groups run concurrently on their own streams,
// single-system groups one after another beside them; the host services
// whichever group's graph has finished.
#include "mrhs.h"
#include "solver.h"

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <map>
#include <memory>
#include <thread>

// Systems on lattices of at least this many 5D sites per checkerboard run
// as groups of one, with the single-system (autotuned) kernels of
// solver.cu inside the same device loop: there a system alone fills the GPU
// and shares too few bytes (the links are 576/Ls of 192 + 576/Ls per site in
// FP32) for lock step to pay (measured at 16^3 x 32 x 16: 8 systems took
// 3.31 s in one group, 2.98 s one after another).
#define MR_SINGLE_SITES (1LL << 19)

// CG iterations per loop body; the residual ring of every batched system
// has this length, so the ring slots and CG-scalar parities baked into the
// body stay valid on every pass (the iteration counter of every system is a
// multiple of MR_BODY whenever the graph starts)
#define MR_BODY 8

// control block of a group (doubles, device): per system the squared
// threshold that sends it to the host, the squared divergence bound, the
// iterations left; outputs: last |r|^2 per system and iterations run
#define CTL_THR 0
#define CTL_RMAX (CTL_THR + MR_MAX)
#define CTL_LEFT (CTL_RMAX + MR_MAX)
#define CTL_RR (CTL_LEFT + MR_MAX)
#define CTL_ITERS (CTL_RR + MR_MAX)
#define CTL_DOUBLES (CTL_ITERS + 8)

namespace {

__global__ void mr_decide_kernel(MRPtrs a, int nr, double* ctl, cudaGraphConditionalHandle h) {
    __shared__ int stop;
    if (threadIdx.x == 0) {
        stop = 0;
        ctl[CTL_ITERS] += (double)MR_BODY;
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (t < nr) {
        const double rr = a.red[t][SC_RRH + (MR_BODY - 1)];
        ctl[CTL_RR + t] = rr;
        const bool bad = !(rr == rr) || rr > 1e300;
        if (bad || rr < ctl[CTL_THR + t] || rr > ctl[CTL_RMAX + t] || ctl[CTL_ITERS] >= ctl[CTL_LEFT + t])
            atomicOr(&stop, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

void mr_dslash(const eofa_ctx* ctx, int prec, int par, int dag, int mode, const MRPtrs& a, const Op5* ops,
               const Op5* ops2, int nr, bool hasop, double a_out, double b_in, int slot, int it, int slot2,
               cudaStream_t st) {
    if (prec == P64) mr_dslash_p64(ctx, par, dag, mode, a, ops, ops2, nr, hasop, a_out, b_in, slot, it, slot2, st);
    else if (prec == P32) mr_dslash_p32(ctx, par, dag, mode, a, ops, ops2, nr, hasop, a_out, b_in, slot, it, slot2, st);
    else mr_dslash_p16(ctx, par, dag, mode, a, ops, ops2, nr, hasop, a_out, b_in, slot, it, slot2, st);
}

void mr_xp(const eofa_ctx* ctx, int prec, const MRPtrs& a, int nr, int it, cudaStream_t st) {
    if (prec == P64) mr_xp_p64(ctx, a, nr, it, st);
    else if (prec == P32) mr_xp_p32(ctx, a, nr, it, st);
    else mr_xp_p16(ctx, a, nr, it, st);
}

struct Group {
    eofa_ctx* ctx = nullptr;
    int prec = 0;
    std::vector<int> members;   // system indices
    std::vector<int> captured;  // active systems baked into the graph
    cudaStream_t st = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    Op5* ops = nullptr;          // device: [Gi x MR_MAX][GiT x MR_MAX] of the captured set
    double* ctl = nullptr;       // device control block
    double* ctl_host = nullptr;  // pinned mirror
    bool single = false;          // one system, single-system kernels
    bool eager_done = false;      // single: the first chunk ran outside a graph (autotuning)
    std::vector<int> last;        // systems of the last launch (graph or eager chunk)
    bool running = false;
    bool finished = false;
    bool pending = false;         // single: waits until the single group before it has finished
    // diagnostics (EOFA_BATCH_LOG=1): host visits, graph builds, host seconds
    int visits = 0, builds = 0;
    double host_s = 0.0, build_s = 0.0;
};

// One lock-step CG iteration (it) of the captured systems: the five fused
// launches of Solve::enqueue, each for all systems at once.
void enqueue_group_iteration(Group& g, std::vector<Solve>& sv, int it, cudaStream_t st) {
    const int n = (int)g.captured.size();
    MRPtrs k1 = {}, k2 = {}, k4 = {}, k5 = {}, k6 = {};
    for (int a = 0; a < n; a++) {
        Solve& s = sv[g.captured[a]];
        k1.in[a] = s.p;  k1.out[a] = s.te; k1.red[a] = s.red;
        k2.in[a] = s.te; k2.out[a] = s.q;  k2.y[a] = s.p;   k2.out2[a] = s.to; k2.red[a] = s.red;
        k4.in[a] = s.to; k4.out[a] = s.te; k4.red[a] = s.red;
        k5.in[a] = s.te; k5.out[a] = s.s;  k5.y[a] = s.q;   k5.out2[a] = s.r; k5.red[a] = s.red;
        k6.out2[a] = s.x; k6.out[a] = s.p; k6.in[a] = s.s;  k6.red[a] = s.red;
    }
    const Op5* Gi = g.ops;
    const Op5* GiT = g.ops + MR_MAX;
    // q = A p: te = G'^-1 D_eo p; q = p - G'^-1 D_oe te, |q|^2 -> delta, to = G'^-T q
    mr_dslash(g.ctx, g.prec, 0, 0, 0, k1, Gi, GiT, n, true, 1.0, 0.0, -1, it, -1, st);
    mr_dslash(g.ctx, g.prec, 1, 0, 1, k2, Gi, GiT, n, true, -1.0, 1.0, SC_DELTA, it, -1, st);
    // s -= alpha A^+ q: te = G'^-T D^+_eo to; s -= alpha (q - D^+_oe te), |s|^2 -> gamma (next
    // parity); r -= alpha q, |r|^2 -> ring
    mr_dslash(g.ctx, g.prec, 0, 1, 0, k4, GiT, GiT, n, true, 1.0, 0.0, -1, it, -1, st);
    mr_dslash(g.ctx, g.prec, 1, 1, 2, k5, GiT, GiT, n, false, -1.0, 1.0, SC_GAMMA + ((it + 1) & 1), it,
              SC_RRH + (it % MR_BODY), st);
    // x += alpha p; p = s + beta p
    mr_xp(g.ctx, g.prec, k6, n, it, st);
}

void destroy_graph(Group& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g.exec = nullptr;
    g.graph = nullptr;
    g.captured.clear();
}

// Graph of the group's device loop for the active set: WHILE(cond) { MR_BODY
// iterations; decide }.
void build_graph(Group& g, std::vector<Solve>& sv, const std::vector<int>& active) {
    auto t0 = std::chrono::steady_clock::now();
    g.builds++;
    destroy_graph(g);
    g.captured = active;
    const int n = (int)active.size();
    std::vector<Op5> h(2 * MR_MAX);
    for (int a = 0; a < n; a++) {
        h[a] = op_finalize(sv[active[a]].Gi, g.ctx->Ls);
        h[MR_MAX + a] = op_finalize(sv[active[a]].GiT, g.ctx->Ls);
    }
    EOFA_CUDA(cudaMemcpyAsync(g.ops, h.data(), h.size() * sizeof(Op5), cudaMemcpyHostToDevice, g.st));
    EOFA_CUDA(cudaStreamSynchronize(g.st));
    EOFA_CUDA(cudaGraphCreate(&g.graph, 0));
    cudaGraphConditionalHandle handle;
    EOFA_CUDA(cudaGraphConditionalHandleCreate(&handle, g.graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    EOFA_CUDA(cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const bool prof_on = g.ctx->prof && g.ctx->prof->on;
    if (g.ctx->prof) g.ctx->prof->on = false;  // no event records inside a conditional body
    try {
        EOFA_CUDA(cudaStreamBeginCaptureToGraph(g.st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        if (g.single) {
            // the single-system launches of Solve::enqueue; the counters it advances
            // are put back (collect_group adds the iterations the loop ran)
            Solve& s1 = sv[active[0]];
            const int it0 = s1.it, n0 = s1.inf.iters;
            s1.enqueue(MR_BODY, g.st);
            s1.it = it0;
            s1.inf.iters = n0;
        } else {
            for (int it = 0; it < MR_BODY; it++) enqueue_group_iteration(g, sv, it, g.st);
        }
        MRPtrs d = {};
        for (int a = 0; a < n; a++) d.red[a] = sv[active[a]].red;
        mr_decide_kernel<<<1, 32, 0, g.st>>>(d, n, g.ctl, handle);
        EOFA_LAUNCHED();
        cudaGraph_t captured = nullptr;
        EOFA_CUDA(cudaStreamEndCapture(g.st, &captured));
    } catch (...) {
        if (g.ctx->prof) g.ctx->prof->on = prof_on;
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(g.st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t gg = nullptr;
            cudaStreamEndCapture(g.st, &gg);
        }
        cudaGetLastError();
        throw;
    }
    if (g.ctx->prof) g.ctx->prof->on = prof_on;
    EOFA_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
    g.build_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Retire, restart or keep the group's systems after a host check; launch the
// device loop for the ones still iterating.  Returns false when every
// system of the group has finished.
bool service_group(Group& g, std::vector<Solve>& sv, std::vector<bool>& finished, std::vector<double*>& xdev) {
    std::vector<int> active;
    for (int i : g.members) {
        if (finished[i]) continue;
        // finish() may ask for a restart (true residual above tol); a restart
        // that is converged at once is finished on the next pass
        for (int pass = 0; pass < 16 && !finished[i]; pass++) {
            if (!(sv[i].done || sv[i].inf.iters >= sv[i].P.maxiter)) break;
            if (sv[i].finish(xdev[i], g.st)) {
                finished[i] = true;
                break;
            }
            sv[i].start_cg(g.st);
        }
        if (!finished[i] && !sv[i].done) active.push_back(i);
    }
    if (active.empty()) {
        // finish() gives up after 8 restarts, so every member is finished here
        for (int i : g.members)
            if (!finished[i]) throw eofa_error(EOFA_EDEVICE, "batched solve: a system neither finished nor active");
        return false;
    }
    g.last = active;
    if (g.single && !g.eager_done) {
        // first chunk outside a graph, so that the autotuner can time the kernel
        // shapes (it does not run during stream capture)
        Solve& s1 = sv[active[0]];
        s1.enqueue(MR_BODY, g.st);
        g.eager_done = true;
        g.ctl_host[CTL_ITERS] = 0.0;  // enqueue advanced the counters itself
        EOFA_CUDA(cudaMemcpyAsync(g.ctl_host + CTL_RR, s1.last_rr(), sizeof(double), cudaMemcpyDeviceToHost, g.st));
        EOFA_CUDA(cudaEventRecord(g.done, g.st));
        g.running = true;
        return true;
    }
    if (!g.exec || active != g.captured) build_graph(g, sv, active);
    for (size_t a = 0; a < active.size(); a++) {
        const Solve& s = sv[active[a]];
        const double thr = s.mixed ? std::max(s.delta * s.rmax, s.target) : s.target;
        g.ctl_host[CTL_THR + a] = thr * thr;
        g.ctl_host[CTL_RMAX + a] = s.mixed ? s.rmax * s.rmax : 1e300;
        g.ctl_host[CTL_LEFT + a] = (double)(s.P.maxiter - s.inf.iters);
    }
    g.ctl_host[CTL_ITERS] = 0.0;
    EOFA_CUDA(cudaMemcpyAsync(g.ctl, g.ctl_host, CTL_DOUBLES * sizeof(double), cudaMemcpyHostToDevice, g.st));
    EOFA_CUDA(cudaGraphLaunch(g.exec, g.st));
    EOFA_CUDA(cudaMemcpyAsync(g.ctl_host + CTL_RR, g.ctl + CTL_RR, (CTL_DOUBLES - CTL_RR) * sizeof(double),
                              cudaMemcpyDeviceToHost, g.st));
    EOFA_CUDA(cudaEventRecord(g.done, g.st));
    g.running = true;
    return true;
}

// The device loop of g has ended: account its iterations and run the host
// checks (reliable updates, convergence) of every captured system.
void collect_group(Group& g, std::vector<Solve>& sv) {
    g.running = false;
    const int n = (int)std::lround(g.ctl_host[CTL_ITERS]);
    for (size_t a = 0; a < g.last.size(); a++) {
        Solve& s = sv[g.last[a]];
        s.it += n;
        s.inf.iters += n;
        s.check_value(g.ctl_host[CTL_RR + a], g.st);
    }
}

}  // namespace

extern "C" int eofa_solve_batched(eofa_ctx* const* ctxs, int n, const eofa_solve_params* params,
                                  const double* const* b, double* const* x, eofa_solve_info* info) {
    if (!ctxs || n < 0 || !params || !b || !x) return EOFA_EINVAL;
    if (n == 0) return EOFA_OK;
    for (int i = 0; i < n; i++)
        if (!ctxs[i] || !b[i] || !x[i]) return EOFA_EINVAL;
    auto t0 = std::chrono::steady_clock::now();
    eofa_ctx* errctx = ctxs[0];
    std::vector<std::unique_ptr<Group>> groups;
    int rc = EOFA_OK;
    try {
        std::vector<Solve> sv(n);
        std::vector<double*> bdev(n), xdev(n);
        std::vector<bool> finished(n, false);
        // groups: same context and inner precision, at most MR_MAX systems each
        std::map<std::pair<eofa_ctx*, int>, Group*> open;
        for (int i = 0; i < n; i++) {
            errctx = ctxs[i];
            const int prec = params[i].precision == EOFA_PREC_F64
                                 ? P64
                                 : (params[i].precision == EOFA_PREC_MIXED_F16 ? P16 : P32);
            auto key = std::make_pair(ctxs[i], prec);
            const bool single = (long long)ctxs[i]->Vh * ctxs[i]->Ls >= MR_SINGLE_SITES;
            Group* g = (!single && open.count(key)) ? open[key] : nullptr;
            if (!g || (int)g->members.size() >= MR_MAX) {
                groups.emplace_back(new Group());
                g = groups.back().get();
                g->ctx = ctxs[i];
                g->prec = prec;
                g->single = single;
                EOFA_CUDA(cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking));
                EOFA_CUDA(cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming));
                const std::string gt = "_g" + std::to_string(groups.size() - 1);
                g->ops = (Op5*)ctx_buffer(g->ctx, "bt_ops" + gt, 2 * MR_MAX * sizeof(Op5));
                g->ctl = (double*)ctx_buffer(g->ctx, "bt_ctl" + gt, CTL_DOUBLES * sizeof(double));
                EOFA_CUDA(cudaMallocHost((void**)&g->ctl_host, CTL_DOUBLES * sizeof(double)));
                open[key] = g;
            }
            g->members.push_back(i);
        }
        for (auto& gp : groups) {
            Group& g = *gp;
            for (int i : g.members) {
                errctx = ctxs[i];
                size_t bytes = (size_t)ctxs[i]->V * ctxs[i]->Ls * 12 * 16;
                std::string tg = "_b" + std::to_string(i);
                bdev[i] = (double*)ctx_buffer(ctxs[i], "bt_b" + tg, bytes);
                xdev[i] = (double*)ctx_buffer(ctxs[i], "bt_x" + tg, bytes);
                double* red = (double*)ctx_buffer(ctxs[i], "bt_red" + tg, red_scratch_bytes());
                EOFA_CUDA(cudaMemsetAsync(red, 0, red_scratch_bytes(), g.st));
                EOFA_CUDA(cudaMemcpyAsync(bdev[i], b[i], bytes, cudaMemcpyHostToDevice, g.st));
                if (params[i].use_x0) EOFA_CUDA(cudaMemcpyAsync(xdev[i], x[i], bytes, cudaMemcpyHostToDevice, g.st));
                sv[i].setup(ctxs[i], params[i], bdev[i], xdev[i], tg, red, MR_BODY, g.st);
                if (!sv[i].trivial) sv[i].start_cg(g.st);
            }
        }
        // Single groups run one at a time, each alone filling the GPU with its
        // fields resident in L2 for its whole device loop, while the lock-step
        // groups of the small lattices run beside them (all single groups at
        // once, 8 systems at 16^3 x 32 x 16 took 3.6 s against 2.7 s for the
        // same solves one after another).
        std::vector<Group*> singles;
        std::map<std::pair<eofa_ctx*, int>, bool> tuned;
        for (auto& gp : groups)
            if (gp->single) {
                gp->pending = !singles.empty();
                singles.push_back(gp.get());
                // the eager first chunk (kernel autotuning, CG form) is needed
                // once per context and precision
                const auto key = std::make_pair(gp->ctx, gp->prec);
                if (tuned[key]) gp->eager_done = true;
                tuned[key] = true;
            }
        // the single groups are the critical path: the host services them first
        std::stable_partition(groups.begin(), groups.end(), [](const std::unique_ptr<Group>& g) { return g->single; });
        size_t next_single = 1;
        auto start_next_single = [&]() {
            while (next_single < singles.size()) {
                Group* ng = singles[next_single++];
                ng->pending = false;
                errctx = ng->ctx;
                ng->finished = !service_group(*ng, sv, finished, xdev);
                if (!ng->finished) break;
            }
        };
        for (auto& gp : groups) {
            // (a single group started by start_next_single is running or finished already)
            if (gp->pending || gp->running || gp->finished) continue;
            errctx = gp->ctx;
            gp->finished = !service_group(*gp, sv, finished, xdev);
            if (gp->single && gp->finished) start_next_single();
        }
        for (;;) {
            bool any = false, progressed = false;
            for (auto& gp : groups) {
                Group& g = *gp;
                if (g.finished) continue;
                any = true;
                if (g.pending || !g.running) continue;
                cudaError_t q = cudaEventQuery(g.done);
                if (q == cudaErrorNotReady) continue;
                EOFA_CUDA(q);
                errctx = g.ctx;
                progressed = true;
                auto th = std::chrono::steady_clock::now();
                g.visits++;
                collect_group(g, sv);
                g.finished = !service_group(g, sv, finished, xdev);
                g.host_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - th).count();
                if (g.single && g.finished) start_next_single();
            }
            if (!any) break;
            if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        for (auto& gp : groups) {
            for (int i : gp->members) {
                errctx = ctxs[i];
                size_t bytes = (size_t)ctxs[i]->V * ctxs[i]->Ls * 12 * 16;
                EOFA_CUDA(cudaMemcpyAsync(x[i], xdev[i], bytes, cudaMemcpyDeviceToHost, gp->st));
            }
            EOFA_CUDA(cudaStreamSynchronize(gp->st));
        }
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (getenv("EOFA_BATCH_LOG"))
            for (size_t k = 0; k < groups.size(); k++)
                fprintf(stderr, "batch group %zu: V=%d Ls=%d prec=%d systems=%zu visits=%d builds=%d host %.3f s (builds %.3f s) of %.3f s\n",
                        k, groups[k]->ctx->V, groups[k]->ctx->Ls, groups[k]->prec, groups[k]->members.size(),
                        groups[k]->visits, groups[k]->builds, groups[k]->host_s, groups[k]->build_s, secs);
        for (int i = 0; i < n; i++) {
            eofa_solve_info inf = sv[i].inf;
            inf.true_resid = sv[i].true_rel;
            inf.seconds = secs;
            inf.status = !std::isfinite(sv[i].true_rel) ? EOFA_ENUMERIC
                                                         : (sv[i].true_rel > sv[i].P.tol ? EOFA_ENOTCONV : EOFA_OK);
            if (info) info[i] = inf;
            if (inf.status != EOFA_OK && rc == EOFA_OK) {
                rc = inf.status;
                ctxs[i]->err = "batched solve " + std::to_string(i) + " did not converge";
            }
        }
    } catch (const eofa_error& e) {
        cudaGetLastError();
        rc = fail(errctx, e.code, e.msg);
    }
    for (auto& gp : groups) {
        Group& g = *gp;
        if (g.st) cudaStreamSynchronize(g.st);
        destroy_graph(g);
        if (g.done) cudaEventDestroy(g.done);
        if (g.ctl_host) cudaFreeHost(g.ctl_host);
    }
    for (auto& gp : groups)
        if (gp->st) cudaStreamDestroy(gp->st);
    return rc;
}
