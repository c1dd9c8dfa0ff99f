// Batches of independent systems (htd_batch_* in include/htd.h).
//
// A batch is a list of instances (handles), instance i carrying nrhs[i]
// right-hand sides.  Every (instance, rhs) pair is one system H_i U = F, solved
// by the same FGMRES(m) as htd_gmres_solve (flexible right preconditioning,
// classical Gram-Schmidt in FP64 with a second pass where the first lost more
// than half of the new vector's norm, Givens
// rotations on the host, true-residual stopping test), but all systems advance
// in lockstep so that the preconditioner applications of one Arnoldi step run
// together:
//
//  - within a handle, one step kernel covers all its active right-hand sides
//    (their slots in the handle's per-rhs arrays; the active list is read by the
//    kernels from device memory, so converged systems drop out of a captured
//    sequence without a new capture);
//  - the 2-D FP32 handles (at least two, Table 1 or exact read-out) run as one
//    persistent launch per run: a queue of (level, instance, rhs slot, tile)
//    tasks of the blocked pair kernel's work, each tile starting a level when
//    its 3 x 3 neighbourhood has finished the previous one (htd_tblock.cu);
//  - the other handles' captured step sequences (different sizes, kernels and
//    step counts T n_P) are child graphs of one graph beside it, launched once
//    per run.
//
// The paper treats one system at a time (Sec. 5); the batch changes only the
// schedule, not the arithmetic of any system.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "htd.h"
#include "htd_internal.h"
#include "htd_krylov_host.h"

typedef std::complex<double> zc;

namespace {

#define HTD_CUDA(x)                                          \
    do {                                                     \
        cudaError_t e_ = (x);                                \
        if (e_ != cudaSuccess) {                             \
            (void)cudaGetLastError();                        \
            return (e_ == cudaErrorMemoryAllocation) ? HTD_ERR_OOM : HTD_ERR_CUDA; \
        }                                                    \
    } while (0)

constexpr int kHBlock = 160;     // double2 per system in the host/device staging buffers

struct Sys {
    int inst = 0, rhs = 0;
    int64_t N = 0;
    int m = 0;
    const double2 *F = nullptr;
    double2 *U = nullptr;
    double2 *V = nullptr, *Z = nullptr, *r = nullptr;   // Krylov workspace
    // FGMRES state
    bool done = false, restart = true;
    int j = 0, its = 0;
    double fnorm = 0.0, bnorm = 0.0;
    std::vector<zc> Hm, cs, g, y;
    std::vector<double> sn;
    htd_solve_info info{};
};

}  // namespace

struct htd_batch_s {
    std::vector<htd_ctx *> ctx;
    std::vector<int> nrhs;
    std::vector<htd::CtxInfo> ci;
    std::vector<Sys> sys;
    std::vector<int> first;              // first system of each instance
    int device = 0;
    double2 *ws = nullptr;               // Krylov workspace of all systems
    double2 *hdev = nullptr, *hhost = nullptr;   // per-system staging blocks
    // per instance, rcap entries each: input and output vector of every rhs slot
    const double2 **tab_host = nullptr;
    const double2 **tab_dev = nullptr;
    std::vector<int64_t> tab_off;        // first entry of instance i (F table; U at + rcap)
    cudaEvent_t tab_ev = nullptr;        // last copy of the table (guards tab_host)
    bool tab_pending = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // two graphs of one run: every handle's step sequence as a child graph
    // (exec_plain), or the group launch beside the other handles' sequences
    // (exec); `form` is the one in use: 0 undecided (the first rounds of a
    // solve time both), 1 plain, 2 group
    cudaGraphExec_t exec = nullptr, exec_plain = nullptr;
    bool graph_tried = false;
    int form = 0;
    int round_form = 0;                  // form of the last round launched
    double form_ms[3] = {0.0, 0.0, 0.0};
    // the persistent launch over the 2-D handles
    std::vector<char> in_group;          // per instance
    std::vector<int> group;              // instance indices, most levels first
    htd::TbPlan gplan{};
    int gctas = 0;
    htd::GroupSched gsched{};
    htd::GroupInst *ginst = nullptr;
    long long *glev = nullptr, *goff = nullptr;
    int *gdone = nullptr, *gabort = nullptr;
    size_t gdone_n = 0;
    unsigned long long *ghead = nullptr;
    float *gab = nullptr;
};

namespace {

void free_batch(htd_batch b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->exec_plain) cudaGraphExecDestroy(b->exec_plain);
    void *gp[] = {b->ginst, b->glev, b->goff, b->gdone, b->gabort, b->ghead, b->gab};
    for (void *q : gp)
        if (q) cudaFree(q);
    if (b->ws) cudaFree(b->ws);
    if (b->hdev) cudaFree(b->hdev);
    if (b->tab_dev) cudaFree(b->tab_dev);
    if (b->hhost) cudaFreeHost(b->hhost);
    if (b->tab_host) cudaFreeHost(b->tab_host);
    if (b->tab_ev) cudaEventDestroy(b->tab_ev);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    delete b;
}

// The group of 2-D handles run by one persistent launch: its instance table
// (tensor maps for the group plan's box, planes, coefficients, step tables),
// the level and instance offsets of the task queue, and the counters.
htd_status build_group(htd_batch b)
{
    const int ninst = (int)b->ctx.size();
    b->in_group.assign(ninst, 0);
    std::vector<htd::CtxGroupView> views(ninst);
    std::vector<int> cand;
    for (int i = 0; i < ninst; ++i)
        if (htd::ctx_group_view(b->ctx[i], &views[i])) cand.push_back(i);
    if (cand.size() < 2 || !htd::group2d_plan(&b->gplan)) return HTD_OK;
    const htd::TbPlan &P = b->gplan;
    b->gctas = htd::group2d_ctas();
    if (b->gctas < 1) return HTD_OK;
    auto nlev = [&](int i) { return (int)((views[i].nsteps + P.B - 1) / P.B); };
    std::stable_sort(cand.begin(), cand.end(), [&](int x, int y) { return nlev(x) > nlev(y); });
    const int ng = (int)cand.size();
    std::vector<htd::GroupInst> gi(ng);
    std::vector<long long> inst_off(ng + 1, 0);
    size_t ab_n = 0, done_n = 0;
    for (int g = 0; g < ng; ++g) {
        const htd::CtxGroupView &v = views[cand[g]];
        ab_n += v.ab.size();
        const int gx = (int)((v.L.nx + P.TX - 1) / P.TX), gy = (int)((v.L.ny + P.TY - 1) / P.TY);
        done_n += (size_t)gx * gy * v.R.slots;
    }
    HTD_CUDA(htd::dev_malloc((void **)&b->gab, sizeof(float) * ab_n));
    HTD_CUDA(htd::dev_malloc((void **)&b->gdone, sizeof(int) * done_n));
    b->gdone_n = done_n;
    size_t ab_at = 0, done_at = 0;
    for (int g = 0; g < ng; ++g) {
        const htd::CtxGroupView &v = views[cand[g]];
        htd::GroupInst &I = gi[g];
        std::memset((void *)&I, 0, sizeof(I));
        float *planes[6] = {v.u[0], v.u[1], v.u[2], v.u[3], const_cast<float *>(v.kap),
                            const_cast<float *>(v.dco)};
        if (!htd::make_tb2d_maps<float>(v.L, P, planes, &I.maps, v.rcap)) {
            (void)cudaGetLastError();
            return HTD_OK;                   // no tensor maps: keep the per-handle launches
        }
        for (int q = 0; q < 4; ++q) I.u[q] = v.u[q];
        I.dco = v.dco;
        I.fre = v.fre;
        I.fim = v.fim;
        I.L = v.L;
        I.C = v.C;
        HTD_CUDA(cudaMemcpy(b->gab + ab_at, v.ab.data(), sizeof(float) * v.ab.size(),
                            cudaMemcpyHostToDevice));
        I.ab = b->gab + ab_at;
        ab_at += v.ab.size();
        I.nsteps = v.nsteps;
        I.jim = v.jim;
        I.jfin = v.jfin;
        I.slot = v.slot;
        I.R = v.R;
        I.err = v.err;
        I.grid_x = (int)((v.L.nx + P.TX - 1) / P.TX);
        I.grid_y = (int)((v.L.ny + P.TY - 1) / P.TY);
        I.nlev = nlev(cand[g]);
        I.done = b->gdone + done_at;
        done_at += (size_t)I.grid_x * I.grid_y * v.R.slots;
        inst_off[g + 1] = inst_off[g] + (long long)I.grid_x * I.grid_y * v.R.slots;
    }
    const int nlev_max = gi[0].nlev;
    std::vector<long long> lev_off(nlev_max + 1, 0);
    for (int k = 0, active = ng; k < nlev_max; ++k) {
        while (active > 0 && gi[active - 1].nlev <= k) --active;
        lev_off[k + 1] = lev_off[k] + inst_off[active];
    }
    HTD_CUDA(htd::dev_malloc((void **)&b->ginst, sizeof(htd::GroupInst) * ng));
    HTD_CUDA(cudaMemcpy(b->ginst, gi.data(), sizeof(htd::GroupInst) * ng, cudaMemcpyHostToDevice));
    HTD_CUDA(htd::dev_malloc((void **)&b->glev, sizeof(long long) * (nlev_max + 1)));
    HTD_CUDA(cudaMemcpy(b->glev, lev_off.data(), sizeof(long long) * (nlev_max + 1),
                        cudaMemcpyHostToDevice));
    HTD_CUDA(htd::dev_malloc((void **)&b->goff, sizeof(long long) * (ng + 1)));
    HTD_CUDA(cudaMemcpy(b->goff, inst_off.data(), sizeof(long long) * (ng + 1),
                        cudaMemcpyHostToDevice));
    HTD_CUDA(htd::dev_malloc((void **)&b->ghead, sizeof(unsigned long long)));
    HTD_CUDA(htd::dev_malloc((void **)&b->gabort, sizeof(int)));
    htd::GroupSched &S = b->gsched;
    S.inst = b->ginst;
    S.lev_off = b->glev;
    S.inst_off = b->goff;
    S.ninst = ng;
    S.nlev_max = nlev_max;
    S.ntasks = lev_off[nlev_max];
    S.head = b->ghead;
    S.abort = b->gabort;
    b->group = cand;
    for (int i : cand) b->in_group[i] = 1;
    return HTD_OK;
}

// one run of the group: every member starts from rest, the queue and the
// counters start at zero, then the persistent launch
htd_status run_group(htd_batch b, cudaStream_t s)
{
    for (int i : b->group) {
        htd_status st = htd::ctx_zero_states(b->ctx[i], s);
        if (st != HTD_OK) return st;
    }
    HTD_CUDA(cudaMemsetAsync(b->gdone, 0, sizeof(int) * b->gdone_n, s));
    HTD_CUDA(cudaMemsetAsync(b->ghead, 0, sizeof(unsigned long long), s));
    HTD_CUDA(cudaMemsetAsync(b->gabort, 0, sizeof(int), s));
    htd::launch_group2d(b->gplan, b->gsched, b->gctas, s);
    HTD_CUDA(cudaGetLastError());
    return HTD_OK;
}

// Instantiate a graph whose children (no dependencies between them, so they
// may run concurrently) are the given graphs.
htd_status make_parent(const std::vector<cudaGraph_t> &kids, cudaGraphExec_t *out)
{
    cudaGraph_t parent = nullptr;
    HTD_CUDA(cudaGraphCreate(&parent, 0));
    bool ok = true;
    for (cudaGraph_t g : kids) {
        cudaGraphNode_t node;
        if (cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, g) != cudaSuccess) {
            ok = false;
            break;
        }
    }
    if (ok && cudaGraphInstantiate(out, parent, 0) != cudaSuccess) {
        *out = nullptr;
        ok = false;
    }
    cudaGraphDestroy(parent);
    (void)cudaGetLastError();
    return HTD_OK;
}

// The batch graphs: every handle's captured step sequence as a child graph
// (the plain form), and, when the batch has a group of 2-D handles, the group
// launch beside the other handles' sequences.  Both give the same bits; the
// first rounds of a solve time them and the faster one is kept.
htd_status build_graph(htd_batch b)
{
    if (b->graph_tried) return HTD_OK;
    b->graph_tried = true;
    htd_status gst = build_group(b);
    if (gst != HTD_OK) return gst;
    std::vector<cudaGraph_t> all, others;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        cudaGraph_t g = htd::ctx_step_graph(b->ctx[i]);
        if (!g) return HTD_OK;               // no capture: run the handles one by one
        all.push_back(g);
        if (!b->in_group[i]) others.push_back(g);
    }
    if ((gst = make_parent(all, &b->exec_plain)) != HTD_OK) return gst;
    if (!b->group.empty()) {
        cudaGraph_t ggraph = nullptr;
        cudaStream_t cs;
        HTD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const long long before = htd::g_launches;
            htd_status st = run_group(b, cs);
            ok = cudaStreamEndCapture(cs, &ggraph) == cudaSuccess && st == HTD_OK;
            htd::g_launches = before;        // captured, not launched
        }
        cudaStreamDestroy(cs);
        (void)cudaGetLastError();
        if (ok) {
            others.push_back(ggraph);
            if ((gst = make_parent(others, &b->exec)) != HTD_OK) return gst;
        }
        if (ggraph) cudaGraphDestroy(ggraph);  // the parent holds its own copy
    }
    if (!b->exec) b->form = 1;               // no group: the plain form only
    return HTD_OK;
}

// Stage every instance's vector table (input Fp[r], output Up[r] of each rhs
// slot) and copy it to the device.  The host table is rewritten only after the
// previous copy has completed.
htd_status upload_table(htd_batch b, cudaStream_t s)
{
    HTD_CUDA(cudaMemcpyAsync(b->tab_dev, b->tab_host, sizeof(double2 *) * b->tab_off.back(),
                             cudaMemcpyHostToDevice, s));
    HTD_CUDA(cudaEventRecord(b->tab_ev, s));
    b->tab_pending = true;
    return HTD_OK;
}

htd_status wait_table(htd_batch b)
{
    if (b->tab_pending) {
        HTD_CUDA(cudaEventSynchronize(b->tab_ev));
        b->tab_pending = false;
    }
    return HTD_OK;
}

// One preconditioner application for the systems with sel[k] set: U_k = P F_k
// (in/out vectors per system given by in[k], out[k]).  Returns the device time
// through the batch events (read later).
htd_status precond_round(htd_batch b, const std::vector<char> &sel,
                         const std::vector<const double2 *> &in, const std::vector<double2 *> &out,
                         cudaStream_t s)
{
    htd::NvtxRange nvtx_range("batch_round");
    const int ninst = (int)b->ctx.size();
    HTD_CUDA(cudaEventRecord(b->ev[0], s));
    htd_status st = wait_table(b);
    if (st != HTD_OK) return st;
    std::vector<std::vector<int>> idx(ninst);
    int runs = 0;
    for (size_t k = 0; k < b->sys.size(); ++k) {
        if (!sel[k]) continue;
        const Sys &y = b->sys[k];
        idx[y.inst].push_back(y.rhs);
        b->tab_host[b->tab_off[y.inst] + y.rhs] = in[k];
        b->tab_host[b->tab_off[y.inst] + b->ci[y.inst].rcap + y.rhs] = out[k];
        runs = std::max(runs, b->ci[y.inst].runs);
    }
    if ((st = upload_table(b, s)) != HTD_OK) return st;
    for (int run = 0; run < runs; ++run) {
        bool any = false;
        for (int i = 0; i < ninst; ++i) {
            const bool on = !idx[i].empty() && run < b->ci[i].runs;
            const double2 *const *Fp = b->tab_dev + b->tab_off[i];
            double2 *const *Up = const_cast<double2 *const *>(b->tab_dev + b->tab_off[i] +
                                                               b->ci[i].rcap);
            st = htd::ctx_stage_run(b->ctx[i], run, on ? (int)idx[i].size() : 0,
                                    on ? idx[i].data() : nullptr, Fp, Up, s);
            if (st != HTD_OK) return st;
            if (on) {
                any = true;
                htd::ctx_account(b->ctx[i], run == 0 ? 1 : 0, b->ci[i].nsteps);
            }
        }
        if (!any) continue;
        // undecided: the plain form first, then the group form
        const int use = (b->form != 0) ? b->form : (b->form_ms[1] == 0.0 ? 1 : 2);
        cudaGraphExec_t ex = (use == 2) ? b->exec : b->exec_plain;
        if (ex) {
            HTD_CUDA(cudaGraphLaunch(ex, s));
            b->round_form = use;
            for (int i = 0; i < ninst; ++i)
                if (use == 1 || !b->in_group[i]) htd::g_launches += b->ci[i].nsteps;
            if (use == 2) htd::g_launches += 1;
        } else {
            b->round_form = 0;
            for (int i = 0; i < ninst; ++i) {
                const bool on = !idx[i].empty() && run < b->ci[i].runs;
                if (!on || b->in_group[i]) continue;
                if ((st = htd::ctx_run_steps(b->ctx[i], s)) != HTD_OK) return st;
            }
            if (!b->group.empty() && (st = run_group(b, s)) != HTD_OK) return st;
        }
    }
    HTD_CUDA(cudaEventRecord(b->ev[1], s));
    return HTD_OK;
}

double round_ms(htd_batch b)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0.0;
    }
    return ms;
}

// squared norms / dots of the listed systems into their staging blocks, one copy
// back, one synchronisation
htd_status fetch_blocks(htd_batch b, cudaStream_t s)
{
    HTD_CUDA(cudaMemcpyAsync(b->hhost, b->hdev, sizeof(double2) * kHBlock * b->sys.size(),
                             cudaMemcpyDeviceToHost, s));
    HTD_CUDA(cudaStreamSynchronize(s));
    HTD_CUDA(cudaGetLastError());
    return HTD_OK;
}

htd_status batch_gmres(htd_batch b, const void *const *F_dev, void *const *U_dev, double tol,
                       int maxit, cudaStream_t s, htd_solve_info *info)
{
    htd::NvtxRange nvtx_range("htd_batch_gmres_solve");
    const auto t0 = std::chrono::steady_clock::now();
    const long long launches0 = htd::g_launches;
    const size_t ns = b->sys.size();
    htd_status st = HTD_OK;
    std::vector<char> sel(ns, 0);
    std::vector<const double2 *> in(ns, nullptr);
    std::vector<double2 *> out(ns, nullptr);
    for (size_t k = 0; k < ns; ++k) {
        Sys &y = b->sys[k];
        y.F = static_cast<const double2 *>(F_dev[y.inst]) + (int64_t)y.rhs * y.N;
        y.U = static_cast<double2 *>(U_dev[y.inst]) + (int64_t)y.rhs * y.N;
        y.done = false;
        y.restart = true;
        y.j = 0;
        y.its = 0;
        std::memset(&y.info, 0, sizeof(y.info));
        y.Hm.assign((size_t)(y.m + 1) * y.m, 0.0);
        y.cs.assign(y.m, 0.0);
        y.sn.assign(y.m, 0.0);
        y.g.assign(y.m + 1, 0.0);
        y.y.assign(y.m, 0.0);
    }
    if ((st = build_graph(b)) != HTD_OK) return st;

    // ||F|| of every system
    for (size_t k = 0; k < ns; ++k) {
        Sys &y = b->sys[k];
        htd::ctx_dots(b->ctx[y.inst], y.F, 0, 1, y.F, b->hdev + k * kHBlock, s);
    }
    if ((st = fetch_blocks(b, s)) != HTD_OK) return st;
    for (size_t k = 0; k < ns; ++k) {
        Sys &y = b->sys[k];
        const double f2 = b->hhost[k * kHBlock].x;
        if (!std::isfinite(f2)) return HTD_ERR_NONFINITE;
        y.fnorm = y.bnorm = std::sqrt(f2 > 0 ? f2 : 0.0);
        if (y.fnorm == 0.0) {
            HTD_CUDA(cudaMemsetAsync(y.U, 0, sizeof(double2) * y.N, s));
            y.done = true;
            y.info.converged = 1;
        }
    }

    for (;;) {
        // ---- cycle starts: true residual r = F - H U, convergence test -----
        bool any_restart = false;
        for (size_t k = 0; k < ns; ++k) {
            Sys &y = b->sys[k];
            if (y.done || !y.restart) continue;
            any_restart = true;
            htd::ctx_apply_H(b->ctx[y.inst], y.U, y.F, y.r, s);
            htd::ctx_dots(b->ctx[y.inst], y.r, 0, 1, y.r, b->hdev + k * kHBlock, s);
        }
        if (any_restart) {
            if ((st = fetch_blocks(b, s)) != HTD_OK) return st;
            for (size_t k = 0; k < ns; ++k) {
                Sys &y = b->sys[k];
                if (y.done || !y.restart) continue;
                const double r2 = b->hhost[k * kHBlock].x;
                if (!std::isfinite(r2)) return HTD_ERR_NONFINITE;
                const double rn = std::sqrt(r2 > 0 ? r2 : 0.0);
                y.info.rel_res_true = rn / y.fnorm;
                if (y.info.rel_res_true <= tol) {
                    y.info.converged = 1;
                    y.done = true;
                    continue;
                }
                if (y.its >= maxit || rn == 0.0) {
                    y.done = true;
                    continue;
                }
                y.info.restarts++;
                htd::launch_scale(y.r, 1.0 / rn, y.V, y.N, s);
                for (int i = 0; i <= y.m; ++i) y.g[i] = 0.0;
                y.g[0] = rn;
                y.j = 0;
                y.restart = false;
            }
        }
        for (size_t k = 0; k < ns; ++k) sel[k] = !b->sys[k].done;
        if (std::none_of(sel.begin(), sel.end(), [](char c) { return c != 0; })) break;

        // ---- Z_j = P V_j for every running system, one graph launch per run --
        for (size_t k = 0; k < ns; ++k) {
            Sys &y = b->sys[k];
            in[k] = y.V + (int64_t)y.j * y.N;
            out[k] = y.Z + (int64_t)y.j * y.N;
        }
        if ((st = precond_round(b, sel, in, out, s)) != HTD_OK) return st;

        // ---- w = H Z_j built in basis slot j + 1, Gram-Schmidt against V_0..V_j:
        // pass 1 for every running system, one fetch; pass 2 for the systems
        // whose first pass lost more than half of ||w||^2 (the single-system
        // driver's test, so both take the same decisions), one more fetch ----
        for (size_t k = 0; k < ns; ++k) {
            if (!sel[k]) continue;
            Sys &y = b->sys[k];
            htd_ctx *c = b->ctx[y.inst];
            const int kc = y.j + 1;
            double2 *vn = y.V + (int64_t)kc * y.N;
            htd::ctx_apply_H(c, y.Z + (int64_t)y.j * y.N, nullptr, vn, s);
            double2 *hb = b->hdev + k * kHBlock;
            htd::ctx_dots(c, y.V, y.N, kc + 1, vn, hb, s);         // V_i^H w and ||w||^2
            htd::launch_sub_combination(y.V, y.N, kc, hb, vn, y.N, s);
        }
        if ((st = fetch_blocks(b, s)) != HTD_OK) return st;
        std::vector<char> second(ns, 0);
        std::vector<double> w1sq(ns, 0.0);
        bool any_second = false;
        for (size_t k = 0; k < ns; ++k) {
            if (!sel[k]) continue;
            Sys &y = b->sys[k];
            second[k] = htd::cgs_needs_second_pass(b->hhost + k * kHBlock, y.j + 1, &w1sq[k]);
            if (!second[k]) continue;
            any_second = true;
            const int kc = y.j + 1;
            double2 *vn = y.V + (int64_t)kc * y.N;
            double2 *hb = b->hdev + k * kHBlock + 72;
            htd::ctx_dots(b->ctx[y.inst], y.V, y.N, kc + 1, vn, hb, s);
            htd::launch_sub_combination(y.V, y.N, kc, hb, vn, y.N, s);
        }
        if (any_second && (st = fetch_blocks(b, s)) != HTD_OK) return st;
        const double ms = round_ms(b);
        if (b->form == 0 && b->round_form != 0) {
            // the form choice: device time per point update of this round
            double upd = 0.0;
            for (size_t k = 0; k < ns; ++k)
                if (sel[k]) {
                    const htd::CtxInfo &ci = b->ci[b->sys[k].inst];
                    upd += (double)b->sys[k].N * (double)ci.nsteps * ci.runs;
                }
            if (upd > 0.0 && ms > 0.0) b->form_ms[b->round_form] = 1e6 * ms / upd;   // ns per update
            if (b->form_ms[1] > 0.0 && b->form_ms[2] > 0.0)
                b->form = (b->form_ms[2] < b->form_ms[1]) ? 2 : 1;
        }

        // ---- Givens update on the host; finished cycles update U -------------
        bool any_y = false;
        for (size_t k = 0; k < ns; ++k) {
            if (!sel[k]) continue;
            Sys &y = b->sys[k];
            const double2 *hh = b->hhost + k * kHBlock;
            const int m = y.m, j = y.j;
            y.info.precond_applies++;
            y.info.steps += b->ci[y.inst].nsteps * b->ci[y.inst].runs;
            y.info.ms_precond += ms;
            zc *col = &y.Hm[(size_t)j * (m + 1)];
            double hn2 = w1sq[k];
            if (second[k]) {
                hn2 = htd::cgs2_column(hh, hh + 72, j + 1, col);
                y.info.reorth++;
            } else {
                htd::cgs1_column(hh, j + 1, col);
            }
            if (!std::isfinite(hn2)) return HTD_ERR_NONFINITE;
            const double hn = std::sqrt(hn2 > 0 ? hn2 : 0.0);
            col[j + 1] = hn;
            double2 *vn = y.V + (int64_t)(j + 1) * y.N;
            if (hn > 0.0) htd::launch_scale(vn, 1.0 / hn, vn, y.N, s);
            htd::givens_column(col, y.cs.data(), y.sn.data(), y.g.data(), j);
            ++y.its;
            ++y.j;
            const double est = std::abs(y.g[y.j]) / y.bnorm;
            y.info.rel_res_est = est;
            if (y.info.hist_len < 256) y.info.hist[y.info.hist_len++] = est;
            if (!std::isfinite(est)) return HTD_ERR_NONFINITE;
            if (est <= tol || y.j == m || y.its >= maxit || hn == 0.0) {
                // y = R^{-1} g; U += Z y
                const int jj = y.j;
                htd::solve_upper(y.Hm.data(), m, y.g.data(), y.y.data(), jj);
                double2 *hy = b->hhost + k * kHBlock;
                for (int i = 0; i < jj; ++i) hy[i] = make_double2(y.y[i].real(), y.y[i].imag());
                HTD_CUDA(cudaMemcpyAsync(b->hdev + k * kHBlock, hy, sizeof(double2) * jj,
                                         cudaMemcpyHostToDevice, s));
                htd::launch_add_combination(y.Z, y.N, jj, b->hdev + k * kHBlock, y.U, y.N, s);
                y.restart = true;
                any_y = true;
            }
        }
        // the staging blocks are rewritten next round: wait for the copies
        if (any_y) HTD_CUDA(cudaStreamSynchronize(s));
    }

    // device error words (bounded waits of the TMA kernels)
    for (htd_ctx *c : b->ctx) {
        htd_status e = htd::ctx_take_error(c);
        if (e != HTD_OK && st == HTD_OK) st = e;
    }
    bool all = true;
    for (Sys &y : b->sys) {
        y.info.iterations = y.its;
        if (!y.info.converged) all = false;
        if (!std::isfinite(y.info.rel_res_true) && st == HTD_OK) st = HTD_ERR_NONFINITE;
    }
    if (st == HTD_OK && !all) st = HTD_ERR_NOT_CONVERGED;
    const double ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) {
        for (size_t k = 0; k < ns; ++k) {
            info[k] = b->sys[k].info;
            info[k].ms_total = ms_total;
            info[k].launches = htd::g_launches - launches0;
        }
    }
    return st;
}

htd_status create_batch(int ninst, const htd_handle *handles, const int *nrhs, htd_batch b)
{
    HTD_CUDA(cudaGetDevice(&b->device));
    size_t ws = 0;
    int64_t tab = 0;
    b->tab_off.push_back(0);
    for (int i = 0; i < ninst; ++i) {
        htd_ctx *c = handles[i];
        if (!c) return HTD_ERR_ARG;
        for (int i2 = 0; i2 < i; ++i2)
            if (handles[i2] == c) return HTD_ERR_ARG;
        htd::CtxInfo ci;
        htd::ctx_info(c, &ci);
        if (ci.device != b->device) return HTD_ERR_ARG;
        if (ci.krylov != HTD_FGMRES) return HTD_ERR_ARG;
        if (nrhs[i] < 1 || nrhs[i] > ci.rcap) return HTD_ERR_ARG;
        b->ctx.push_back(c);
        b->nrhs.push_back(nrhs[i]);
        b->ci.push_back(ci);
        b->first.push_back((int)b->sys.size());
        for (int r = 0; r < nrhs[i]; ++r) {
            Sys y;
            y.inst = i;
            y.rhs = r;
            y.N = ci.N;
            y.m = ci.m;
            b->sys.push_back(y);
            ws += (size_t)(2 * ci.m + 2) * (size_t)ci.N;
        }
        tab += 2 * ci.rcap;
        b->tab_off.push_back(tab);
    }
    for (htd_ctx *c : b->ctx) htd::ctx_join_batch(c);
    HTD_CUDA(htd::dev_malloc((void **)&b->ws, sizeof(double2) * ws));
    size_t off = 0;
    for (Sys &y : b->sys) {
        y.V = b->ws + off;
        off += (size_t)(y.m + 1) * y.N;
        y.Z = b->ws + off;
        off += (size_t)y.m * y.N;
        y.r = b->ws + off;
        off += (size_t)y.N;
    }
    const size_t hb = sizeof(double2) * kHBlock * b->sys.size();
    HTD_CUDA(htd::dev_malloc((void **)&b->hdev, hb));
    HTD_CUDA(cudaMemset(b->hdev, 0, hb));
    HTD_CUDA(htd::host_malloc((void **)&b->hhost, hb));
    HTD_CUDA(htd::dev_malloc((void **)&b->tab_dev, sizeof(double2 *) * tab));
    HTD_CUDA(cudaMemset(b->tab_dev, 0, sizeof(double2 *) * tab));
    HTD_CUDA(htd::host_malloc((void **)&b->tab_host, sizeof(double2 *) * tab));
    std::memset(b->tab_host, 0, sizeof(double2 *) * tab);
    HTD_CUDA(cudaEventCreateWithFlags(&b->tab_ev, cudaEventDisableTiming));
    HTD_CUDA(cudaEventCreate(&b->ev[0]));
    HTD_CUDA(cudaEventCreate(&b->ev[1]));
    return HTD_OK;
}

}  // namespace

extern "C" {

htd_status htd_batch_describe(htd_batch b, htd_batch_desc *out)
{
    if (!b || !out) return HTD_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    out->instances = (int)b->ctx.size();
    out->systems = (int)b->sys.size();
    if (!b->group.empty()) {
        out->grouped = (int)b->group.size();
        out->group_ctas = b->gctas;
        out->group_tasks = b->gsched.ntasks;
        out->group_steps_per_task = b->gplan.B;
    }
    out->form = b->form;
    out->ns_per_update_plain = b->form_ms[1];
    out->ns_per_update_group = b->form_ms[2];
    return HTD_OK;
}

htd_status htd_batch_set_form(htd_batch b, int form)
{
    if (!b || form < 0 || form > 2) return HTD_ERR_ARG;
    htd_status st = build_graph(b);
    if (st != HTD_OK) return st;
    if (form == 2 && !b->exec) return HTD_ERR_ARG;
    if (form == 1 && !b->exec_plain) return HTD_ERR_ARG;
    b->form = form;
    if (form == 0) b->form_ms[1] = b->form_ms[2] = 0.0;
    return HTD_OK;
}

htd_status htd_batch_create(int ninst, const htd_handle *handles, const int *nrhs, htd_batch *out)
{
    if (!out || !handles || !nrhs || ninst < 1) return HTD_ERR_ARG;
    htd_batch b = new (std::nothrow) htd_batch_s();
    if (!b) return HTD_ERR_OOM;
    htd_status st = create_batch(ninst, handles, nrhs, b);
    if (st != HTD_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return HTD_OK;
}

htd_status htd_batch_destroy(htd_batch b)
{
    if (!b) return HTD_OK;
    cudaDeviceSynchronize();
    free_batch(b);
    return HTD_OK;
}

htd_status htd_batch_apply_precond(htd_batch b, const void *const *F_dev, void *const *U_dev,
                                   void *stream)
{
    if (!b || !F_dev || !U_dev) return HTD_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (!F_dev[i] || !U_dev[i] || F_dev[i] == U_dev[i]) return HTD_ERR_ARG;
    htd_status st = build_graph(b);
    if (st != HTD_OK) return st;
    const size_t ns = b->sys.size();
    std::vector<char> sel(ns, 1);
    std::vector<const double2 *> in(ns);
    std::vector<double2 *> out(ns);
    for (size_t k = 0; k < ns; ++k) {
        const Sys &y = b->sys[k];
        in[k] = static_cast<const double2 *>(F_dev[y.inst]) + (int64_t)y.rhs * y.N;
        out[k] = static_cast<double2 *>(U_dev[y.inst]) + (int64_t)y.rhs * y.N;
    }
    return precond_round(b, sel, in, out, s);
}

htd_status htd_batch_gmres_solve(htd_batch b, const void *const *F_dev, void *const *U_dev,
                                 double tol, int max_iters, void *stream, htd_solve_info *info)
{
    if (!b || !F_dev || !U_dev || max_iters < 0 || !(tol > 0.0)) return HTD_ERR_ARG;
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (!F_dev[i] || !U_dev[i] || F_dev[i] == U_dev[i]) return HTD_ERR_ARG;
    return batch_gmres(b, F_dev, U_dev, tol, max_iters, static_cast<cudaStream_t>(stream), info);
}

}  // extern "C"
