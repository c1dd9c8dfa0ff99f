// C ABI of libhtd (declared in include/htd.h): problem set-up, parameter
// selection, the preconditioner driver and the restarted (F)GMRES driver.
// Method: C. C. Stolk, "A time-domain preconditioner for the Helmholtz
// equation" (arXiv 2006.16861).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "htd.h"
#include "htd_internal.h"
#include "htd_krylov_host.h"

using htd::Layout;
using htd::OutSlot;
using htd::StepCoef;
typedef std::complex<double> zc;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxRestart = 64;
// streamed 3-D step kernels: shapes 0..2 one node per thread (32 x 8, 64 x 4,
// 128 x 2 tiles), 3 = node pairs in paired FP32 instructions (64 x 8 tiles)
constexpr int kS3Pair = 3;
constexpr int kS3Default = kS3Pair;

// ---------------------------------------------------------------------------
// stencil weights per Hamming distance (App. A cell form, h = 1)
// ---------------------------------------------------------------------------

// Q1 elements factor into 1-D element matrices per axis: stiffness
// k1 = [[1,-1],[-1,1]], consistent mass m1 = [[1/3,1/6],[1/6,1/3]].  For two
// corners differing on s axes the d-D entries are
//   stiffness: sum over axes of k1 on that axis times m1 on the others,
//   consistent mass: prod of m1.
// Q1MIX mass = half consistent + half lumped (2^-d on the diagonal).
// FD5: each grid edge shared by 2^{d-1} cells carries weight w = 2^{1-d}, so a
// corner has stiffness d w and its edge neighbours -w; lumped mass 2^-d.
// FAMILY(a, gamma): gamma Q1 stiffness + (1 - gamma) FD5 stiffness, a
// consistent mass + (1 - a) lumped mass (Q1MIX = (0.5, 1), FD5 = (0, 0)).
bool cell_weights(int d, int stencil, double a, double gamma, double S[4], double M[4])
{
    for (int s = 0; s < 4; ++s) { S[s] = 0.0; M[s] = 0.0; }
    if (stencil == HTD_STENCIL_Q1MIX) {
        a = 0.5;
        gamma = 1.0;
    } else if (stencil == HTD_STENCIL_FD5) {
        a = 0.0;
        gamma = 0.0;
    } else if (stencil != HTD_STENCIL_FAMILY || !(a >= 0.0 && a <= 1.0) ||
               !(gamma >= 0.0 && gamma <= 1.0)) {
        return false;
    }
    const double m_same = 1.0 / 3.0, m_diff = 1.0 / 6.0;
    const double w = std::ldexp(1.0, 1 - d);
    for (int s = 0; s <= d; ++s) {
        // Q1: axes that differ contribute k1 = -1 (and m1 = 1/6 when not differentiated)
        double q1 = 0.0;
        q1 += s * (-1.0) * std::pow(m_diff, s - 1) * std::pow(m_same, d - s);
        q1 += (d - s) * (1.0) * std::pow(m_diff, s) * std::pow(m_same, d - s - 1);
        const double fd = (s == 0) ? d * w : (s == 1) ? -w : 0.0;
        S[s] = (gamma == 1.0) ? q1 : (gamma == 0.0) ? fd : gamma * q1 + (1.0 - gamma) * fd;
        const double cons = std::pow(m_diff, s) * std::pow(m_same, d - s);
        const double lump = (s == 0) ? std::ldexp(1.0, -d) : 0.0;
        M[s] = (a == 0.0) ? lump : a * cons + (1.0 - a) * lump;
    }
    return true;
}

double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// Eigenvalue of a Hamming-distance kernel f_s on {0,1}^d for Walsh functions
// of weight w: sum_s f_s K_s(w), K_s the Krawtchouk polynomial.  2^d times it
// is the constant-coefficient symbol at the vertex of [0,pi]^d with w
// coordinates equal to pi.
double walsh_eigen(int d, const double f[4], int w)
{
    double mu = 0.0;
    for (int s = 0; s <= d; ++s) {
        double K = 0.0;
        for (int j = 0; j <= s; ++j) K += ((j & 1) ? -1.0 : 1.0) * binom(w, j) * binom(d - w, s - j);
        mu += f[s] * K;
    }
    return mu;
}

// sine-squared window of the paper (Sec. 2.3), even, 1 on |s| <= 1 - rho
double window_chi(double s, double rho)
{
    s = std::fabs(s);
    if (s >= 1.0) return 0.0;
    if (s <= 1.0 - rho) return 1.0;
    const double v = std::sin(0.5 * kPi * (1.0 - s) / rho);
    return v * v;
}

Layout make_layout(int d, const int64_t n[3], size_t esz)
{
    Layout L;
    L.d = d;
    L.nx = n[d - 1];
    L.ny = n[d - 2];
    L.nz = (d == 3) ? n[0] : 1;
    const int64_t line = 128 / (int64_t)esz;       // elements per 128 bytes
    L.xl = line;
    L.pitch = ((L.xl + L.nx + 1 + line - 1) / line) * line;
    L.plane = L.pitch * (L.ny + 2);
    L.total = (d == 3) ? L.plane * (L.nz + 2) : L.plane;
    L.N = L.nx * L.ny * L.nz;
    return L;
}

}  // namespace

struct htd_ctx {
    int device = 0;
    htd_options opt{};
    int d = 0;
    int64_t n[3] = {1, 1, 1};
    double h = 0, omega_phys = 0;
    // parameters
    double kmin = 0, kmax = 0, omega = 0, lam_reH = 0, lam_A = 0, dt = 0, alpha = 0, beta = 0, rho = 0;
    int nP = 0, T = 0;
    long long nsteps = 0;
    double S[4] = {0}, M[4] = {0};
    Layout Lr{}, L64{};
    size_t esz = 8;
    // recurrence arrays (element type float or double)
    void *kap = nullptr, *dco = nullptr, *fre = nullptr, *fim = nullptr, *u0 = nullptr, *u1 = nullptr;
    std::vector<double> atab, btab;
    StepCoef<double> C{};
    // FP64 operator data
    double *kap64 = nullptr, *imH = nullptr;
    double *coefP = nullptr;    // assembled operator, h_planes(d) planes of N
    double *coefI = nullptr;    // assembled Im H (cell damping only), same layout
    // Krylov workspace
    int m = 20;
    double2 *V = nullptr, *Z = nullptr, *w = nullptr, *t = nullptr, *r = nullptr;
    double2 *partial = nullptr, *hdev = nullptr, *hhost = nullptr;
    int nb = 1;
    OutSlot *slot = nullptr;
    double2 *Fh = nullptr, *Uh = nullptr;
    // temporally blocked path (2-D, FP32): second pair of state planes
    void *u2 = nullptr, *u3 = nullptr;
    htd::TbPlan tb{};
    htd::TbMaps tbmaps{};
    bool use_tb = false;
    // resident-grid 2-D step (FP32, one rhs): a whole run in one cooperative launch
    htd::Res2dPlan res{};
    bool use_res = false;
    void *res_ab = nullptr;                 // a_j, b_j per step, in the recurrence precision
    void *res_w = nullptr;                  // projection weights per phase (PROJECT)
    unsigned long long *res_x = nullptr;    // edge exchange buffer
    // TMA-streamed 3-D step (FP32)
    htd::Stream3Maps s3maps{};
    bool use_s3 = false;
    int s3_zchunk = 0;
    int s3_shape = 0;
    int s3_stages = 5;
    int s3_rpc = 1;             // right-hand sides per CTA of the streamed pair kernel
    // right-hand-side batch: rcap rhs slots in every per-rhs array (u0, u1, u2,
    // u3, fre, fim, slot); act_dev = active list read by the step kernels
    int rcap = 1;
    int *act_dev = nullptr;
    // projection read-out: 4 planes of N per rhs (sums and compensations, re/im)
    void *acc = nullptr;
    htd::RhsSet Rs{};
    int *err_dev = nullptr;     // set by a kernel whose bounded device wait gave up
    float step_us = 0.f;        // autotuned time per recurrence step (microseconds)
    // gradient workspace (htd_grad), allocated on first use
    double2 *gU = nullptr, *gMu = nullptr, *gR = nullptr, *gres = nullptr;
    int64_t *grec = nullptr;
    int grec_cap = 0;
    // htd_grad_td workspace (checkpoints, segment states, multipliers), grown on demand
    void *td_ws = nullptr;
    size_t td_ws_bytes = 0;
    // captured step sequence
    cudaGraph_t graph = nullptr;          // kept for batches (child graph nodes)
    cudaGraphExec_t exec = nullptr;
    bool graph_tried = false;
    long long steps_run = 0;
    int applies = 0;
    // device time of preconditioner applications (CUDA events on the call's stream)
    cudaEvent_t pev[2] = {nullptr, nullptr};
    bool pev_pending = false;
    double ms_precond = 0.0;
};

namespace {

#define HTD_CUDA(x)                                          \
    do {                                                     \
        cudaError_t e_ = (x);                                \
        if (e_ != cudaSuccess) {                             \
            (void)cudaGetLastError();                        \
            return (e_ == cudaErrorMemoryAllocation) ? HTD_ERR_OOM : HTD_ERR_CUDA; \
        }                                                    \
    } while (0)

template <typename T>
StepCoef<T> cast_coef(const StepCoef<double> &c)
{
    StepCoef<T> o;
    o.c0 = (T)c.c0;
    for (int k = 0; k < 4; ++k) { o.cs[k] = (T)c.cs[k]; o.mt[k] = (T)c.mt[k]; }
    return o;
}

void free_ctx(htd_ctx *c)
{
    if (!c) return;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    for (cudaEvent_t e : c->pev)
        if (e) cudaEventDestroy(e);
    void *dev[] = {c->kap, c->dco, c->fre, c->fim, c->u0, c->u1, c->kap64, c->imH, c->coefP, c->coefI, c->V, c->Z,
                   c->w, c->t, c->r, c->partial, c->hdev, c->slot, c->Fh, c->Uh, c->u2, c->u3,
                   c->err_dev, c->gU, c->gMu, c->gR, c->gres, c->grec, c->act_dev,
                   c->acc, c->td_ws, c->res_ab, c->res_x, c->res_w};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (c->hhost) cudaFreeHost(c->hhost);
    delete c;
}

// Consecutive launches of the blocked 2-D and the streamed 3-D step overlap
// (programmatic dependent launch) unless the handle's options say
// HTD_LAUNCH_NO_OVERLAP.
bool step_overlap(const htd_ctx *c)
{
    return !(c->opt.launch & HTD_LAUNCH_NO_OVERLAP);
}

// One preconditioner run of T n_P steps; the forcing planes are already filled.
// Table 1 / EXACT: the step kernels write the snapshot and final state into the
// output slots (flags).  PROJECT: steps j >= j_acc (whose new states u_{j+1}
// lie in the last proj_periods periods) run one step per launch, each
// followed by the compensated accumulation of e^{-i theta_{j+1}} u_{j+1};
// a finishing kernel writes (2 / n_acc) times the sums to the output slots.
template <typename T>
htd_status run_steps_direct(htd_ctx *c, cudaStream_t s)
{
    const Layout &L = c->Lr;
    const StepCoef<T> C = cast_coef<T>(c->C);
    const bool project = c->opt.mode == HTD_MODE_PROJECT;
    const long long jim = project ? -1 : c->nsteps - c->nP / 4;
    const long long jfin = project ? -1 : c->nsteps;
    if (c->use_res) {
        // the whole run in one launch; the global state planes are not used.
        // PROJECT: the kernel accumulates the window's states itself, then the
        // finishing kernel writes (2 / n_acc) times the sums
        htd::Res2dProj<T> P;
        const long long n_res = project ? (long long)c->opt.proj_periods * c->nP : 0;
        if (project) {
            P.j_acc = (int)(c->nsteps - n_res);
            P.nP = c->nP;
            P.w = (const T *)c->res_w;
            P.acc = (T *)c->acc;
            P.N = L.N;
            HTD_CUDA(cudaMemsetAsync(c->acc, 0, sizeof(T) * 4 * L.N, s));
        }
        htd::launch_res2d<T>(c->res, (const T *)c->kap, (const T *)c->dco, (const T *)c->fre,
                             (const T *)c->fim, L, C, (const T *)c->res_ab, (int)c->nsteps,
                             (int)jim, (int)jfin, c->slot, c->res_x, c->err_dev, s, P);
        if (project)
            htd::launch_project_finish<T>(L.N, (const T *)c->acc, 4 * L.N, 2.0 / (double)n_res,
                                          c->slot, c->Rs, s);
        HTD_CUDA(cudaGetLastError());
        return HTD_OK;
    }
    T *A = (T *)c->u0, *B = (T *)c->u1;
    HTD_CUDA(cudaMemsetAsync(A, 0, sizeof(T) * L.total * c->rcap, s));
    HTD_CUDA(cudaMemsetAsync(B, 0, sizeof(T) * L.total * c->rcap, s));
    const long long n_acc = project ? (long long)c->opt.proj_periods * c->nP : 0;
    const long long j_acc = c->nsteps - n_acc;           // first step whose new state counts
    const int64_t astride = 4 * L.N;
    if (project) HTD_CUDA(cudaMemsetAsync(c->acc, 0, sizeof(T) * astride * c->rcap, s));
    // accumulate the new state u_{j+1} (in `u`) of step j
    auto accumulate = [&](long long j, const T *u) {
        const double th = 2.0 * kPi * (double)((j + 1) % c->nP) / (double)c->nP;
        htd::launch_project_accumulate<T>(L, u, (T *)c->acc, astride, (T)std::cos(th),
                                          (T)(-std::sin(th)), c->Rs, s);
    };
    auto finish = [&]() {
        htd::launch_project_finish<T>(L.N, (const T *)c->acc, astride, 2.0 / (double)n_acc,
                                      c->slot, c->Rs, s);
    };
    // one-step launches for steps j0 .. nsteps-1 from (cur = u_{j0}, oth = u_{j0-1})
    auto one_steps = [&](long long j0, T *cur, T *oth) {
        for (long long j = j0; j < c->nsteps; ++j) {
            int flags = 0;
            if (j + 1 == jim) flags |= 1;
            if (j + 1 == jfin) flags |= 2;
            htd::launch_step<T>(L, cur, oth, (const T *)c->kap, (const T *)c->dco,
                                (const T *)c->fre, (const T *)c->fim, C, (T)c->atab[j],
                                (T)c->btab[j], c->slot, flags, s, c->Rs);
            if (project && j >= j_acc) accumulate(j, oth);
            std::swap(cur, oth);
        }
    };
    if (c->opt.integrator == HTD_ABD) {
        // backward differences: u_{j+1} into a third plane (the cell-damping term
        // reads u_{j-1} at the neighbours)
        T *cur = A, *prv = B, *nxt = (T *)c->u2;
        const T cth = (T)std::cos(2.0 * kPi / (double)c->nP);
        const bool cell = c->opt.damping == HTD_DAMP_CELL;
        for (long long j = 0; j < c->nsteps; ++j) {
            int flags = 0;
            if (j + 1 == jim) flags |= 1;
            if (j + 1 == jfin) flags |= 2;
            htd::launch_abd_step<T>(L, cur, prv, nxt, (const T *)c->kap, (const T *)c->dco, cell,
                                    (const T *)c->fre, (const T *)c->fim, C, (T)c->atab[j],
                                    (T)c->btab[j], cth, c->slot, flags, s, c->Rs);
            if (project && j >= j_acc) accumulate(j, nxt);
            T *t = prv;
            prv = cur;
            cur = nxt;
            nxt = t;
        }
        if (project) finish();
        HTD_CUDA(cudaGetLastError());
        return HTD_OK;
    }
    if constexpr (std::is_same<T, float>::value) {
      if (c->use_tb) {
        // B steps per launch; the state pair alternates between (u0,u1) and (u2,u3)
        T *pairs[2][2] = {{A, B}, {(T *)c->u2, (T *)c->u3}};
        const int map_of[2][2] = {{0, 1}, {2, 3}};
        const long long jend = project ? j_acc : c->nsteps;   // blocked steps end here
        int from = 0;
        for (long long j0 = 0; j0 < jend; j0 += c->tb.B) {
            htd::TbSteps<T> S;
            S.nsub = (int)std::min<long long>(c->tb.B, jend - j0);
            for (int q = 0; q < htd::kTbMaxSteps; ++q) {
                const long long j = j0 + q;
                S.a[q] = (q < S.nsub) ? (T)c->atab[j] : T(0);
                S.b[q] = (q < S.nsub) ? (T)c->btab[j] : T(0);
                int flags = 0;
                if (q < S.nsub && j + 1 == jim) flags |= 1;
                if (q < S.nsub && j + 1 == jfin) flags |= 2;
                S.flags[q] = flags;
            }
            htd::launch_tb2d<T>(c->tb, c->tbmaps, map_of[from][0], map_of[from][1], L,
                                pairs[1 - from][0], pairs[1 - from][1], (const T *)c->dco,
                                (const T *)c->fre, (const T *)c->fim, C, S, c->slot,
                                c->err_dev, s, c->Rs, j0 > 0 && step_overlap(c));
            from = 1 - from;
        }
        // the blocked launches leave u_{jend} in pairs[from][0], u_{jend-1} in pairs[from][1]
        if (project) {
            one_steps(jend, pairs[from][0], pairs[from][1]);
            finish();
        }
        HTD_CUDA(cudaGetLastError());
        return HTD_OK;
      }
    }
    if constexpr (std::is_same<T, float>::value) {
        if (c->use_s3) {
            for (long long j = 0; j < c->nsteps; ++j) {
                int flags = 0;
                if (j + 1 == jim) flags |= 1;
                if (j + 1 == jfin) flags |= 2;
                T *um = (j & 1) ? A : B;                    // receives u_{j+1}
                if (c->s3_shape == kS3Pair)
                    htd::launch_stream3d_pair(c->s3maps, (int)(j & 1), L, um, C,
                                              (T)c->atab[j], (T)c->btab[j], c->slot, flags,
                                              c->s3_zchunk, c->s3_stages, c->err_dev, s, c->Rs,
                                              j > 0 && step_overlap(c), c->s3_rpc);
                else
                    htd::launch_stream3d(c->s3maps, (int)(j & 1), c->s3_shape, L, um, C,
                                         (T)c->atab[j], (T)c->btab[j], c->slot, flags,
                                         c->s3_zchunk, c->err_dev, s);
                if (project && j >= j_acc) accumulate(j, um);
            }
            if (project) finish();
            HTD_CUDA(cudaGetLastError());
            return HTD_OK;
        }
    }
    one_steps(0, A, B);
    if (project) finish();
    HTD_CUDA(cudaGetLastError());
    return HTD_OK;
}

// HTD_LAUNCH_NO_GRAPH: the steps are launched one by one instead of replaying
// a captured graph
bool graphs_disabled(const htd_ctx *c)
{
    return (c->opt.launch & HTD_LAUNCH_NO_GRAPH) != 0;
}

// Capture the whole step sequence of one run into a graph (once per handle):
// c->graph keeps it (a batch adds it as a child graph), c->exec replays it.
template <typename T>
void capture_steps(htd_ctx *c)
{
    if (c->graph_tried) return;
    c->graph_tried = true;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        const long long before = htd::g_launches;
        htd_status st = run_steps_direct<T>(c, cs);
        ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && st == HTD_OK;
        htd::g_launches = before;            // captured, not launched
    }
    if (ok && cudaGraphInstantiate(&c->exec, g, 0) != cudaSuccess) {
        c->exec = nullptr;
        ok = false;
    }
    if (ok) {
        c->graph = g;
        g = nullptr;
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    (void)cudaGetLastError();
}

template <typename T>
htd_status run_steps(htd_ctx *c, cudaStream_t s)
{
    if (!graphs_disabled(c)) capture_steps<T>(c);
    if (c->exec) {
        HTD_CUDA(cudaGraphLaunch(c->exec, s));
        htd::g_launches += c->nsteps;            // one step kernel per graph node
        return HTD_OK;
    }
    return run_steps_direct<T>(c, s);
}

// add the elapsed time of the last timed preconditioner application
htd_status collect_precond_time(htd_ctx *c)
{
    if (!c->pev_pending) return HTD_OK;
    HTD_CUDA(cudaEventSynchronize(c->pev[1]));
    float ms = 0.f;
    HTD_CUDA(cudaEventElapsedTime(&ms, c->pev[0], c->pev[1]));
    c->ms_precond += ms;
    c->pev_pending = false;
    return HTD_OK;
}

// U = P F (F, U compact complex128 on the device)
htd_status precond(htd_ctx *c, const double2 *F, double2 *U, cudaStream_t s)
{
    htd::NvtxRange nvtx_range("precond");
    const bool mixed = c->opt.precision == HTD_MIXED;
    htd_status cst = collect_precond_time(c);
    if (cst != HTD_OK) return cst;
    HTD_CUDA(cudaEventRecord(c->pev[0], s));
    const int only0 = 0;
    htd::launch_set_act(c->act_dev, 1, &only0, s);       // one rhs: slot 0 -> rhs 0
    double *Ure = reinterpret_cast<double *>(U);
    const int runs = (c->opt.mode == HTD_MODE_EXACT) ? 2 : 1;
    for (int run = 0; run < runs; ++run) {
        // TABLE1: final state -> Re U, quarter-period-earlier snapshot -> Im U.
        // EXACT: run 0 forcing F gives Re S_T F; run 1 forcing -iF gives Im S_T F.
        if (mixed)
            htd::launch_split<float>(c->Lr, F, (float *)c->fre, (float *)c->fim, run, s);
        else
            htd::launch_split<double>(c->Lr, F, (double *)c->fre, (double *)c->fim, run, s);
        double *fin = Ure + run;
        double *snap = (runs == 1) ? Ure + 1 : nullptr;
        htd::launch_set_slot(c->slot, fin, snap, s);
        HTD_CUDA(cudaGetLastError());
        htd_status st = mixed ? run_steps<float>(c, s) : run_steps<double>(c, s);
        if (st != HTD_OK) return st;
        c->steps_run += c->nsteps;
    }
    HTD_CUDA(cudaEventRecord(c->pev[1], s));
    c->pev_pending = true;
    c->applies++;
    return HTD_OK;
}

void apply_H(htd_ctx *c, const double2 *X, const double2 *F, double2 *Y, cudaStream_t s)
{
    htd::launch_apply_H(c->L64, c->coefP, c->imH, 1.0 / (c->h * c->h), X, F, Y, s, c->coefI);
}

// dots of w with V_0..V_{k-1} into hdev + off (device); does not synchronise
void dots_to(htd_ctx *c, const double2 *V, int k, const double2 *w, int off, cudaStream_t s)
{
    const int64_t N = c->Lr.N;
    htd::launch_dots(V, N, k, w, N, c->partial, c->nb, s);
    htd::launch_reduce(c->partial, c->nb, k, c->hdev + off, s);
}

// ||x|| (synchronises)
htd_status norm(htd_ctx *c, const double2 *x, double *out, cudaStream_t s)
{
    dots_to(c, x, 1, x, 0, s);
    HTD_CUDA(cudaMemcpyAsync(c->hhost, c->hdev, sizeof(double2), cudaMemcpyDeviceToHost, s));
    HTD_CUDA(cudaStreamSynchronize(s));
    const double v = c->hhost[0].x;
    if (!std::isfinite(v)) return HTD_ERR_NONFINITE;
    *out = std::sqrt(v > 0 ? v : 0.0);
    return HTD_OK;
}

htd_status gmres(htd_ctx *c, const double2 *F, double2 *U, double tol, int maxit, cudaStream_t s,
                 htd_solve_info *info)
{
    const auto t0 = std::chrono::steady_clock::now();
    const int64_t N = c->Lr.N;
    const int m = c->m;
    const bool left = c->opt.krylov == HTD_LEFT_GMRES;
    const bool fixed = !(tol > 0.0);
    htd_solve_info loc;
    std::memset(&loc, 0, sizeof(loc));
    const int applies0 = c->applies;
    const long long steps0 = c->steps_run;
    const long long launches0 = htd::g_launches;
    if (collect_precond_time(c) != HTD_OK) return HTD_ERR_CUDA;
    const double msp0 = c->ms_precond;
    htd_status st = HTD_OK;
    double fnorm = 0.0, bnorm = 0.0;
    std::vector<zc> Hm((size_t)(m + 1) * m), cs(m), g(m + 1), y(m);
    std::vector<double> sn(m);
    int its = 0;

    if ((st = norm(c, F, &fnorm, s)) != HTD_OK) goto out;
    if (fnorm == 0.0) {
        HTD_CUDA(cudaMemsetAsync(U, 0, sizeof(double2) * N, s));
        HTD_CUDA(cudaStreamSynchronize(s));
        loc.converged = 1;
        goto out;
    }
    bnorm = fnorm;
    if (left) {
        if ((st = precond(c, F, c->t, s)) != HTD_OK) goto out;
        if ((st = norm(c, c->t, &bnorm, s)) != HTD_OK) goto out;
        if (bnorm == 0.0) { st = HTD_ERR_NONFINITE; goto out; }
    }
    for (;;) {
        // true residual r = F - H U
        apply_H(c, U, F, c->r, s);
        double rn;
        if ((st = norm(c, c->r, &rn, s)) != HTD_OK) goto out;
        loc.rel_res_true = rn / fnorm;
        if (!fixed && loc.rel_res_true <= tol) { loc.converged = 1; break; }
        if (its >= maxit) break;
        const double2 *r0 = c->r;
        if (left) {
            if ((st = precond(c, c->r, c->w, s)) != HTD_OK) goto out;
            r0 = c->w;
        }
        double beta;
        if ((st = norm(c, r0, &beta, s)) != HTD_OK) goto out;
        if (beta == 0.0) break;
        loc.restarts++;
        htd::launch_scale(r0, 1.0 / beta, c->V, N, s);
        for (int k = 0; k <= m; ++k) g[k] = 0.0;
        g[0] = beta;
        int j = 0;
        while (j < m && its < maxit) {
            double2 *vj = c->V + (int64_t)j * N;
            double2 *vn = c->V + (int64_t)(j + 1) * N;     // the new vector, built in place
            if (!left) {
                double2 *zj = c->Z + (int64_t)j * N;
                if ((st = precond(c, vj, zj, s)) != HTD_OK) goto out;
                apply_H(c, zj, nullptr, vn, s);
            } else {
                apply_H(c, vj, nullptr, c->t, s);
                if ((st = precond(c, c->t, vn, s)) != HTD_OK) goto out;
            }
            // classical Gram-Schmidt, FP64: per pass V_i^H w for i <= j and
            // ||w||^2 in one kernel, then w -= V h; a second pass only when the
            // first lost more than half of ||w||^2 (cgs_needs_second_pass)
            const int k = j + 1;
            dots_to(c, c->V, k + 1, vn, 0, s);
            htd::launch_sub_combination(c->V, N, k, c->hdev, vn, N, s);
            HTD_CUDA(cudaMemcpyAsync(c->hhost, c->hdev, sizeof(double2) * (k + 1),
                                     cudaMemcpyDeviceToHost, s));
            HTD_CUDA(cudaStreamSynchronize(s));
            HTD_CUDA(cudaGetLastError());
            zc *col = &Hm[(size_t)j * (m + 1)];
            double hn2 = 0.0;
            if (htd::cgs_needs_second_pass(c->hhost, k, &hn2)) {
                dots_to(c, c->V, k + 1, vn, 72, s);
                htd::launch_sub_combination(c->V, N, k, c->hdev + 72, vn, N, s);
                HTD_CUDA(cudaMemcpyAsync(c->hhost + 72, c->hdev + 72, sizeof(double2) * (k + 1),
                                         cudaMemcpyDeviceToHost, s));
                HTD_CUDA(cudaStreamSynchronize(s));
                HTD_CUDA(cudaGetLastError());
                hn2 = htd::cgs2_column(c->hhost, c->hhost + 72, k, col);
                ++loc.reorth;
            } else {
                htd::cgs1_column(c->hhost, k, col);
            }
            if (!std::isfinite(hn2)) { st = HTD_ERR_NONFINITE; goto out; }
            const double hn = std::sqrt(hn2 > 0 ? hn2 : 0.0);
            col[j + 1] = hn;
            if (hn > 0.0) htd::launch_scale(vn, 1.0 / hn, vn, N, s);
            // previous rotations, then a new one zeroing col[j+1]
            htd::givens_column(col, cs.data(), sn.data(), g.data(), j);
            ++its;
            ++j;
            const double est = std::abs(g[j]) / bnorm;
            loc.rel_res_est = est;
            if (loc.hist_len < 256) loc.hist[loc.hist_len++] = est;
            if (!std::isfinite(est)) { st = HTD_ERR_NONFINITE; goto out; }
            if (!fixed && est <= tol) break;
            if (hn == 0.0) break;
        }
        // y = R^{-1} g; U += basis y
        htd::solve_upper(Hm.data(), m, g.data(), y.data(), j);
        for (int i = 0; i < j; ++i) c->hhost[i] = make_double2(y[i].real(), y[i].imag());
        HTD_CUDA(cudaMemcpyAsync(c->hdev, c->hhost, sizeof(double2) * j, cudaMemcpyHostToDevice, s));
        htd::launch_add_combination(left ? c->V : c->Z, N, j, c->hdev, U, N, s);
        // the host staging buffer is reused: wait for the copy before the next write
        HTD_CUDA(cudaStreamSynchronize(s));
    }
    if (!fixed && !loc.converged) st = HTD_ERR_NOT_CONVERGED;
    if (!std::isfinite(loc.rel_res_true)) st = HTD_ERR_NONFINITE;
out:
    if (collect_precond_time(c) != HTD_OK && st == HTD_OK) st = HTD_ERR_CUDA;
    {
        // a bounded device-side wait that gave up makes the whole result invalid
        int flag = 0;
        if (cudaMemcpy(&flag, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            (void)cudaGetLastError();
            if (st == HTD_OK) st = HTD_ERR_CUDA;
        } else if (flag) {
            cudaMemset(c->err_dev, 0, sizeof(int));
            st = HTD_ERR_TIMEOUT;
        }
    }
    loc.ms_precond = c->ms_precond - msp0;
    loc.launches = htd::g_launches - launches0;
    loc.iterations = its;
    loc.precond_applies = c->applies - applies0;
    loc.steps = c->steps_run - steps0;
    loc.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = loc;
    return st;
}

template <typename T>
htd_status upload_recurrence(htd_ctx *c, const std::vector<double> &qkap, const std::vector<double> &dcoef)
{
    const Layout &L = c->Lr;
    std::vector<T> a(L.total, (T)0), b(L.total, (T)0);
    for (size_t i = 0; i < (size_t)L.total; ++i) { a[i] = (T)qkap[i]; b[i] = (T)dcoef[i]; }
    HTD_CUDA(cudaMemcpy(c->kap, a.data(), sizeof(T) * L.total, cudaMemcpyHostToDevice));
    HTD_CUDA(cudaMemcpy(c->dco, b.data(), sizeof(T) * L.total, cudaMemcpyHostToDevice));
    return HTD_OK;
}

// The resident-grid kernel for a single-rhs handle with Table 1 or exact
// read-out whose grid fits: one whole run untimed, one timed; kept when
// `force` or when faster per step than c->step_us (the best so far).
template <typename T>
htd_status try_res2d(htd_ctx *c, bool force, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1)
{
    if (c->rcap != 1 || c->nsteps >= (1LL << 30)) return HTD_OK;
    if (!htd::res2d_plan<T>(c->Lr, &c->res)) return HTD_OK;
    if (c->opt.mode == HTD_MODE_PROJECT) {
        // projection weights per phase k of the new state: cos and -sin of
        // 2 pi k / nP, rounded as for the separate accumulation kernel
        std::vector<T> w(2 * (size_t)c->nP);
        for (int k = 0; k < c->nP; ++k) {
            const double th = 2.0 * kPi * (double)k / (double)c->nP;
            w[2 * k] = (T)std::cos(th);
            w[2 * k + 1] = (T)(-std::sin(th));
        }
        HTD_CUDA(htd::dev_malloc(&c->res_w, sizeof(T) * w.size()));
        HTD_CUDA(cudaMemcpy(c->res_w, w.data(), sizeof(T) * w.size(), cudaMemcpyHostToDevice));
    }
    std::vector<T> ab(2 * (size_t)c->nsteps);
    for (long long j = 0; j < c->nsteps; ++j) {
        ab[2 * j] = (T)c->atab[j];
        ab[2 * j + 1] = (T)c->btab[j];
    }
    HTD_CUDA(htd::dev_malloc(&c->res_ab, sizeof(T) * ab.size()));
    HTD_CUDA(cudaMemcpy(c->res_ab, ab.data(), sizeof(T) * ab.size(), cudaMemcpyHostToDevice));
    HTD_CUDA(htd::dev_malloc(&c->res_x, sizeof(unsigned long long) * c->res.xwords));
    const StepCoef<T> C = cast_coef<T>(c->C);
    for (int r = 0; r < 2; ++r) {
        if (r == 1) HTD_CUDA(cudaEventRecord(e0, s));
        htd::launch_res2d<T>(c->res, (const T *)c->kap, (const T *)c->dco, (const T *)c->fre,
                             (const T *)c->fim, c->Lr, C, (const T *)c->res_ab, (int)c->nsteps,
                             -1, -1, c->slot, c->res_x, c->err_dev, s);
    }
    HTD_CUDA(cudaEventRecord(e1, s));
    HTD_CUDA(cudaEventSynchronize(e1));
    HTD_CUDA(cudaGetLastError());
    float ms = 0.f;
    HTD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    const float us = 1e3f * ms / (float)c->nsteps;
    if (force || us < c->step_us) {
        c->use_res = true;
        c->step_us = us;
    } else {
        cudaFree(c->res_ab);
        cudaFree(c->res_x);
        cudaFree(c->res_w);
        c->res_ab = nullptr;
        c->res_x = nullptr;
        c->res_w = nullptr;
    }
    return HTD_OK;
}

// The plain FP64 2-D recurrence: the one-step kernel (one launch per step)
// against the FP64 resident-grid kernel, each timed on the handle's own
// (zeroed) planes; the faster is kept (HTD_TB_RESIDENT: the resident kernel
// whenever it qualifies).
htd_status autotune_fp64_2d(htd_ctx *c)
{
    cudaStream_t s;
    HTD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    HTD_CUDA(cudaEventCreate(&e0));
    HTD_CUDA(cudaEventCreate(&e1));
    const StepCoef<double> C = cast_coef<double>(c->C);
    const int reps = 64;
    for (int r = 0; r < 2 + reps; ++r) {
        if (r == 2) HTD_CUDA(cudaEventRecord(e0, s));
        htd::launch_step<double>(c->Lr, (const double *)c->u0, (double *)c->u1,
                                 (const double *)c->kap, (const double *)c->dco,
                                 (const double *)c->fre, (const double *)c->fim, C, 0.0, 0.0,
                                 c->slot, 0, s);
    }
    HTD_CUDA(cudaEventRecord(e1, s));
    HTD_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    HTD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    c->step_us = 1e3f * ms / reps;
    htd_status st = try_res2d<double>(c, c->opt.tb_form == HTD_TB_RESIDENT, s, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (st != HTD_OK) return st;
    int flag = 0;
    HTD_CUDA(cudaMemcpy(&flag, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    return flag ? HTD_ERR_TIMEOUT : HTD_OK;
}

// Time the one-step kernel, every blocked configuration and, for a single-rhs
// handle whose grid fits the SMs' shared memory (Table 1 or EXACT read-out),
// the resident-grid kernel on the handle's own (zeroed) planes, and keep the
// fastest per step.  HTD_TB_RESIDENT takes the resident kernel whenever it
// fits; the best blocked configuration is kept as well (a batch uses it).  No
// output is written: the step flags are zero during tuning.
htd_status autotune_tb2d(htd_ctx *c, int want_B, int want_RPT)
{
    const Layout &L = c->Lr;
    std::vector<htd::TbPlan> all = htd::tb2d_candidates<float>(L, want_B);
    std::vector<htd::TbPlan> cands;
    const int form = c->opt.tb_form;                       // HTD_TB_ANY: every form
    const int bform = (form == HTD_TB_RESIDENT) ? HTD_TB_ANY : form;
    for (const htd::TbPlan &p : all) {
        const int pf = !p.pair ? HTD_TB_COLUMN : (p.sd ? HTD_TB_PAIR_SD : HTD_TB_PAIR);
        if ((want_RPT == 0 || p.RPT == want_RPT) && (bform == HTD_TB_ANY || bform == pf))
            cands.push_back(p);
    }
    if (cands.empty()) return HTD_OK;
    const size_t bytes = sizeof(float) * (size_t)L.total * c->rcap;
    HTD_CUDA(htd::dev_malloc(&c->u2, bytes));
    HTD_CUDA(cudaMemset(c->u2, 0, bytes));
    HTD_CUDA(htd::dev_malloc(&c->u3, bytes));
    HTD_CUDA(cudaMemset(c->u3, 0, bytes));
    cudaStream_t s;
    HTD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    HTD_CUDA(cudaEventCreate(&e0));
    HTD_CUDA(cudaEventCreate(&e1));
    const StepCoef<float> C = cast_coef<float>(c->C);
    float *planes[6] = {(float *)c->u0, (float *)c->u1, (float *)c->u2, (float *)c->u3,
                        (float *)c->kap, (float *)c->dco};
    const int reps = 4;
    // the one-step kernel
    float best_us = INFINITY;
    {
        for (int r = 0; r < 2 + reps * 4; ++r) {
            if (r == 2) HTD_CUDA(cudaEventRecord(e0, s));
            htd::launch_step<float>(L, (const float *)c->u0, (float *)c->u1, (const float *)c->kap,
                                    (const float *)c->dco, (const float *)c->fre,
                                    (const float *)c->fim, C, 0.f, 0.f, c->slot, 0, s);
        }
        HTD_CUDA(cudaEventRecord(e1, s));
        HTD_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        HTD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best_us = 1e3f * ms / (reps * 4);
    }
    const float one_step_us = best_us;
    if (want_B > 0) best_us = INFINITY;     // a requested block depth is always used
    int best = -1;
    htd::TbMaps best_maps{};
    for (size_t k = 0; k < cands.size(); ++k) {
        htd::TbMaps maps;
        if (!htd::make_tb2d_maps<float>(L, cands[k], planes, &maps, c->rcap)) continue;
        htd::TbSteps<float> S;
        S.nsub = cands[k].B;
        for (int q = 0; q < htd::kTbMaxSteps; ++q) { S.a[q] = 0.f; S.b[q] = 0.f; S.flags[q] = 0; }
        for (int r = 0; r < 2 + reps; ++r) {
            if (r == 2) HTD_CUDA(cudaEventRecord(e0, s));
            htd::launch_tb2d<float>(cands[k], maps, 0, 1, L, (float *)c->u2, (float *)c->u3,
                                    (const float *)c->dco, (const float *)c->fre,
                                    (const float *)c->fim, C, S, c->slot, c->err_dev, s,
                                    htd::RhsSet{}, r > 0 && step_overlap(c));
        }
        HTD_CUDA(cudaEventRecord(e1, s));
        HTD_CUDA(cudaEventSynchronize(e1));
        HTD_CUDA(cudaGetLastError());
        float ms = 0.f;
        HTD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const float us = 1e3f * ms / (reps * cands[k].B);
        cands[k].us_per_step = us;
        if (us < best_us) {
            best_us = us;
            best = (int)k;
            best_maps = maps;
        }
    }
    c->step_us = (best >= 0) ? best_us : one_step_us;
    if (best >= 0) {
        c->use_tb = true;
        c->tb = cands[best];
        c->tbmaps = best_maps;
    }
    // the resident-grid kernel
    const bool res_try = want_B == 0 && want_RPT == 0 && (form == HTD_TB_ANY || form == HTD_TB_RESIDENT);
    if (res_try) {
        htd_status rs = try_res2d<float>(c, form == HTD_TB_RESIDENT, s, e0, e1);
        if (rs != HTD_OK) return rs;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    int flag = 0;
    HTD_CUDA(cudaMemcpy(&flag, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return HTD_ERR_TIMEOUT;
    return HTD_OK;
}

// z-chunk length of the streamed 3-D step, chosen by timing: every chunk count k
// whose chunk length ceil(nz / k) lies in [16, 128] (nz itself when nz < 16),
// one step each on the context's own buffers with zero forcing and no outputs.
// How the CTAs of the last wave fill the GPU decides the best length, which no
// simple rule predicts well (at 256^3: 37 planes beats 32 and 64 by 3-8 %).
htd_status autotune_s3_zchunk(htd_ctx *c, const htd::RhsSet &R = htd::RhsSet{})
{
    const Layout &L = c->Lr;
    std::vector<int> cands;
    for (int64_t k = 1; k <= L.nz; ++k) {
        const int64_t zc = (L.nz + k - 1) / k;
        if (zc > 128) continue;
        if (zc < 16 && !cands.empty()) break;
        if (cands.empty() || cands.back() != (int)zc) cands.push_back((int)zc);
        if (zc < 16) break;
    }
    if (cands.size() < 2) {
        if (!cands.empty()) c->s3_zchunk = cands[0];
        return HTD_OK;
    }
    cudaStream_t s;
    HTD_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    HTD_CUDA(cudaEventCreate(&e0));
    HTD_CUDA(cudaEventCreate(&e1));
    const StepCoef<float> C = cast_coef<float>(c->C);
    const int reps = 4;
    float best_us = INFINITY;
    int best = c->s3_zchunk;
    // two passes over the candidates, each candidate's best kept: neighbouring
    // chunk lengths differ by 1-2 %, about the spread of a single timing
    for (int pass = 0; pass < 2; ++pass)
    for (int zc : cands) {
        for (int r = 0; r < 2 + reps; ++r) {
            if (r == 2) HTD_CUDA(cudaEventRecord(e0, s));
            if (c->s3_shape == kS3Pair)
                htd::launch_stream3d_pair(c->s3maps, r & 1, L, (r & 1) ? (float *)c->u0
                                                                        : (float *)c->u1,
                                          C, 0.f, 0.f, c->slot, 0, zc, c->s3_stages, c->err_dev, s,
                                          R, r > 0 && step_overlap(c), c->s3_rpc);
            else
                htd::launch_stream3d(c->s3maps, r & 1, c->s3_shape, L,
                                     (r & 1) ? (float *)c->u0 : (float *)c->u1, C, 0.f, 0.f,
                                     c->slot, 0, zc, c->err_dev, s);
        }
        HTD_CUDA(cudaEventRecord(e1, s));
        HTD_CUDA(cudaEventSynchronize(e1));
        HTD_CUDA(cudaGetLastError());
        float ms = 0.f;
        HTD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const float us = 1e3f * ms / reps;
        if (us < best_us) {
            best_us = us;
            best = zc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    int flag = 0;
    HTD_CUDA(cudaMemcpy(&flag, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return HTD_ERR_TIMEOUT;
    c->s3_zchunk = best;
    c->step_us = best_us;
    return HTD_OK;
}

// Misfit of the preconditioner's own output and its gradient through the
// recurrence (htd_grad_td).  Per source: U = P F by the handle's fast path for
// the misfit; then per real run a forward pass of one-step launches that keeps
// (u_j, u_{j-1}) every C steps, and a backward sweep over the segments from the
// last: recompute the segment's states from its checkpoint, run the adjoint
// recurrence (the same step kernel on the multipliers, forcing -dJ/du_k at the
// read-out steps) and add each step's gradient term.  Memory: 2 ceil(N/C) +
// C + 6 planes.
template <typename T>
htd_status grad_td_impl(htd_ctx *c, int nsrc, const double2 *F, int nrec, const double2 *d,
                        int ckpt, double *gm, double *gR, double *misfit, cudaStream_t s)
{
    const Layout &L = c->Lr;
    const int64_t N = L.N;
    const long long ns = c->nsteps;
    const long long jim = ns - c->nP / 4;
    const int runs = (c->opt.mode == HTD_MODE_EXACT) ? 2 : 1;
    const long long C = ckpt > 0 ? std::min<long long>(ckpt, ns)
                                 : std::max<long long>(1, (long long)std::ceil(std::sqrt(2.0 * ns)));
    const long long nseg = (ns + C - 1) / C;
    const size_t plane = sizeof(T) * (size_t)L.total;
    const size_t nplanes = (size_t)(2 * nseg + C + 2 + 2 + 2);
    const size_t need = plane * nplanes + sizeof(double2) * (size_t)N;
    if (need > c->td_ws_bytes) {
        if (c->td_ws) cudaFree(c->td_ws);
        c->td_ws = nullptr;
        c->td_ws_bytes = 0;
        HTD_CUDA(htd::dev_malloc(&c->td_ws, need));
        c->td_ws_bytes = need;
    }
    T *base = static_cast<T *>(c->td_ws);
    auto P = [&](size_t k) { return base + k * (size_t)L.total; };
    T *ck = P(0);                                   // checkpoint m: planes 2m (u_{mC}), 2m+1 (u_{mC-1})
    T *seg = P(2 * nseg);                           // u_{s0-2+i} in plane i, i = 0 .. C+1
    T *lam0 = P(2 * nseg + C + 2), *lam1 = P(2 * nseg + C + 3);
    T *are = P(2 * nseg + C + 4), *aim = P(2 * nseg + C + 5);
    double2 *U = reinterpret_cast<double2 *>(P(nplanes));
    auto seg_of = [&](long long i, long long s0) { return seg + (size_t)(i - s0 + 2) * L.total; };
    HTD_CUDA(cudaMemsetAsync(c->td_ws, 0, plane * nplanes, s));   // ghost rings stay zero
    const StepCoef<T> Cf = cast_coef<T>(c->C);
    const double cK = c->dt * c->dt / c->alpha;
    const double cm = -cK * c->omega_phys * c->omega_phys;
    const double cR = c->beta * c->dt / (2.0 * c->alpha * c->omega) * c->omega_phys;
    const htd::RhsSet one{};
    std::vector<double2> res(nrec > 0 ? nrec : 1);
    double J = 0.0;
    auto step = [&](const T *u, T *um, const T *fre, const T *fim, T a, T b) {
        htd::launch_step<T>(L, u, um, (const T *)c->kap, (const T *)c->dco, fre, fim, Cf, a, b,
                            c->slot, 0, s, one);
    };
    for (int src = 0; src < nsrc; ++src) {
        const double2 *Fs = F + (size_t)src * N;
        htd_status st = precond(c, Fs, U, s);
        if (st != HTD_OK) return st;
        HTD_CUDA(cudaMemsetAsync(are, 0, 2 * plane, s));     // are, aim adjacent
        if (nrec > 0) {
            htd::launch_residual_planes<T>(L, U, d + (size_t)src * nrec, c->grec, nrec, c->gres,
                                           are, aim, s);
            HTD_CUDA(cudaGetLastError());
            HTD_CUDA(cudaMemcpyAsync(res.data(), c->gres, sizeof(double2) * nrec,
                                     cudaMemcpyDeviceToHost, s));
            HTD_CUDA(cudaStreamSynchronize(s));
            for (int k = 0; k < nrec; ++k) J += 0.5 * (res[k].x * res[k].x + res[k].y * res[k].y);
        }
        if (!gm && !gR) continue;
        for (int run = 0; run < runs; ++run) {
            // the run's forcing planes (Table 1: F; EXACT run 1: -iF)
            htd::launch_split<T>(L, Fs, (T *)c->fre, (T *)c->fim, run, s);
            // forward, keeping (u_j, u_{j-1}) at j = m C
            T *cur = seg, *oth = seg + L.total;
            HTD_CUDA(cudaMemsetAsync(seg, 0, 2 * plane, s));
            for (long long j = 0; j < ns; ++j) {
                if (j % C == 0) {
                    const long long m = j / C;
                    HTD_CUDA(cudaMemcpyAsync(P(2 * m), cur, plane, cudaMemcpyDeviceToDevice, s));
                    HTD_CUDA(cudaMemcpyAsync(P(2 * m + 1), oth, plane, cudaMemcpyDeviceToDevice, s));
                }
                step(cur, oth, (const T *)c->fre, (const T *)c->fim, (T)c->atab[j], (T)c->btab[j]);
                std::swap(cur, oth);
            }
            // backward over the segments [s0, s1], s0 = 1 + m C
            HTD_CUDA(cudaMemsetAsync(lam0, 0, 2 * plane, s));     // lam_{k+1}, lam_{k+2}
            T *la = lam0, *lb = lam1;
            for (long long m = nseg - 1; m >= 0; --m) {
                const long long s0 = 1 + m * C, s1 = std::min(s0 + C - 1, ns);
                HTD_CUDA(cudaMemcpyAsync(seg_of(s0 - 2, s0), P(2 * m + 1), plane,
                                         cudaMemcpyDeviceToDevice, s));
                HTD_CUDA(cudaMemcpyAsync(seg_of(s0 - 1, s0), P(2 * m), plane,
                                         cudaMemcpyDeviceToDevice, s));
                for (long long j = s0 - 1; j < s1; ++j) {
                    T *dst = seg_of(j + 1, s0);
                    HTD_CUDA(cudaMemcpyAsync(dst, seg_of(j - 1, s0), plane,
                                             cudaMemcpyDeviceToDevice, s));
                    step(seg_of(j, s0), dst, (const T *)c->fre, (const T *)c->fim, (T)c->atab[j],
                         (T)c->btab[j]);
                }
                for (long long k = s1; k >= s0; --k) {
                    // forcing -dJ/du_k: Table 1 reads Re U at N and Im U at jim; EXACT
                    // reads Re U (run 0) or Im U (run 1) at N
                    T a = T(0), b = T(0);
                    if (runs == 1) {
                        if (k == ns) a = T(-1);
                        if (k == jim) b = T(1);
                    } else if (k == ns) {
                        if (run == 0) a = T(-1); else b = T(1);
                    }
                    step(la, lb, are, aim, a, b);          // lb <- lam_k
                    std::swap(la, lb);                     // la = lam_k, lb = lam_{k+1}
                    htd::launch_grad_td<T>(L, c->M, cm, cR, la, seg_of(k, s0), seg_of(k - 1, s0),
                                           seg_of(k - 2, s0), gm, gR, s);
                }
            }
            HTD_CUDA(cudaGetLastError());
        }
    }
    HTD_CUDA(cudaStreamSynchronize(s));
    *misfit = J;
    return std::isfinite(J) ? HTD_OK : HTD_ERR_NONFINITE;
}

// Host-only validation and parameter selection (Sec. 2.2, App. A).
struct Plan {
    htd_options opt;
    int d = 0;
    int64_t n[3] = {1, 1, 1};
    int64_t N = 1, Nc = 1;
    double S[4], M[4];
    htd_params p;
};

htd_status plan_impl(const htd_grid *grid, const double *c_cell, const double *R_node,
                     double omega_phys, int bc, const htd_options *optp, Plan *pl)
{
    htd_options opt;
    if (optp) opt = *optp; else htd_default_options(&opt);
    if (!grid || !c_cell || !R_node) return HTD_ERR_ARG;
    if (grid->ndim != 2 && grid->ndim != 3) return HTD_ERR_ARG;
    if (!(grid->h > 0.0) || !std::isfinite(grid->h)) return HTD_ERR_ARG;
    if (!(omega_phys > 0.0) || !std::isfinite(omega_phys)) return HTD_ERR_ARG;
    if (bc != HTD_BC_DIRICHLET) return HTD_ERR_ARG;
    if (opt.precision != HTD_FP64 && opt.precision != HTD_MIXED) return HTD_ERR_ARG;
    if (opt.mode != HTD_MODE_TABLE1 && opt.mode != HTD_MODE_EXACT && opt.mode != HTD_MODE_PROJECT)
        return HTD_ERR_ARG;
    if (opt.krylov != HTD_FGMRES && opt.krylov != HTD_LEFT_GMRES) return HTD_ERR_ARG;
    if (opt.T < 1 || !(opt.rho >= 0.0 && opt.rho <= 1.0) || opt.nP < 0) return HTD_ERR_ARG;
    if (opt.restart < 1 || opt.restart > kMaxRestart) return HTD_ERR_ARG;
    if (opt.max_rhs == 0) opt.max_rhs = 1;
    if (opt.max_rhs < 1 || opt.max_rhs > htd::kMaxRhs) return HTD_ERR_ARG;
    if (opt.proj_periods == 0) opt.proj_periods = 1;
    if (opt.proj_periods < 1 || opt.proj_periods > opt.T) return HTD_ERR_ARG;
    if (opt.integrator != HTD_ACD && opt.integrator != HTD_ABD) return HTD_ERR_ARG;
    if (opt.damping != HTD_DAMP_NODE && opt.damping != HTD_DAMP_CELL) return HTD_ERR_ARG;
    // I_acd inverts I + L/2: explicit only for diagonal damping (Sec. 6)
    if (opt.integrator == HTD_ACD && opt.damping == HTD_DAMP_CELL) return HTD_ERR_ARG;
    const int d = grid->ndim;
    pl->d = d;
    pl->N = 1;
    pl->Nc = 1;
    for (int a = 0; a < 3; ++a) pl->n[a] = 1;
    // every product is checked against the node limit before it is formed, so
    // no int64 product can overflow (N <= 2^34 and each factor <= 2^24 + 1)
    constexpr int64_t kMaxNodes = (int64_t)1 << 34;
    for (int a = 0; a < d; ++a) {
        if (grid->n[a] < 1 || grid->n[a] > ((int64_t)1 << 24)) return HTD_ERR_ARG;
        if (pl->N > kMaxNodes / grid->n[a]) return HTD_ERR_ARG;
        if (pl->Nc > (2 * kMaxNodes) / (grid->n[a] + 1)) return HTD_ERR_ARG;
        pl->n[a] = grid->n[a];
        pl->N *= grid->n[a];
        pl->Nc *= grid->n[a] + 1;
    }
    if (!cell_weights(d, opt.stencil, opt.stencil_a, opt.stencil_gamma, pl->S, pl->M))
        return HTD_ERR_ARG;
    if (opt.tblock != 0 && opt.tblock != 1 && opt.tblock != 4 && opt.tblock != 8)
        return HTD_ERR_ARG;
    if (opt.tb_rows != 0 && opt.tb_rows != 6 && opt.tb_rows != 8 && opt.tb_rows != 10 &&
        opt.tb_rows != 12 && opt.tb_rows != 20)
        return HTD_ERR_ARG;
    if (opt.tb_form < HTD_TB_ANY || opt.tb_form > HTD_TB_RESIDENT) return HTD_ERR_ARG;
    if (opt.s3_kernel < HTD_S3_PAIR || opt.s3_kernel > HTD_S3_NODE_128x2) return HTD_ERR_ARG;
    if (opt.s3_stages != 0 && (opt.s3_stages < 4 || opt.s3_stages > 7)) return HTD_ERR_ARG;
    if (opt.s3_zchunk < 0 || opt.s3_zchunk > (1 << 24)) return HTD_ERR_ARG;
    if (opt.s3_rhs_per_cta < 0 || opt.s3_rhs_per_cta > 2) return HTD_ERR_ARG;
    if (opt.launch & ~(HTD_LAUNCH_NO_OVERLAP | HTD_LAUNCH_NO_GRAPH | HTD_LAUNCH_NO_GROUP))
        return HTD_ERR_ARG;
    if (opt.wait_limit_ns < 0) return HTD_ERR_ARG;
    pl->opt = opt;

    double kmin = INFINITY, kmax = 0.0;
    for (int64_t i = 0; i < pl->Nc; ++i) {
        const double cv = c_cell[i];
        if (!std::isfinite(cv)) return HTD_ERR_NONFINITE;
        if (!(cv > 0.0)) return HTD_ERR_ARG;
        const double k = omega_phys / cv;
        kmin = std::fmin(kmin, k);
        kmax = std::fmax(kmax, k);
    }
    double rmax = 0.0;
    for (int64_t i = 0; i < pl->N; ++i) {
        if (!std::isfinite(R_node[i])) return HTD_ERR_NONFINITE;
        if (R_node[i] < 0.0) return HTD_ERR_ARG;
        rmax = std::fmax(rmax, R_node[i]);
    }
    htd_params &P = pl->p;
    P.k_min = kmin;
    P.k_max = kmax;
    P.omega_c = kmax;                              // omega = sqrt(-lambda_min) >= k_max bound
    const double kap_min = (grid->h * kmin) * (grid->h * kmin);
    double f[4];
    for (int s = 0; s < 4; ++s) f[s] = pl->S[s] - kap_min * pl->M[s];
    double lmax = -INFINITY;
    for (int w = 0; w <= d; ++w) lmax = std::fmax(lmax, std::ldexp(walsh_eigen(d, f, w), d));
    P.lam_max_reH = lmax / (grid->h * grid->h);
    P.lam_max_A = P.lam_max_reH + P.omega_c * P.omega_c;
    const double ratio = P.omega_c * P.omega_c / P.lam_max_A;
    int nP = 0;
    if (opt.integrator == HTD_ABD) {
        // Sec. 6.1: theta = omega dt = 2 pi / n_P; omega^2 = k_max^2 + (beta/theta)
        // (1 - cos theta) lambda_max(Im H) makes K >= 0 (App. A: -lambda_min(Re H)
        // <= k_max^2; lambda_max(Im H) <= omega_phys max R for either damping
        // form); n_P is the smallest multiple of 4 with 4 I - K - 2 L > 0 by
        // the scalar bound of Eq. Deltat_bd_full_inequality.
        const double lam_im = omega_phys * rmax;
        auto ok = [&](int q, double *w2) {
            const double th = 2.0 * kPi / q;
            const double al = th * th / (2.0 - 2.0 * std::cos(th)), be = th / std::sin(th);
            *w2 = kmax * kmax + be / th * (1.0 - std::cos(th)) * lam_im;
            const double lhs = th * th / al * (P.lam_max_reH / *w2 + 1.0) +
                               be / al * (1.0 + std::cos(th)) * lam_im / *w2;
            return lhs < 4.0;
        };
        double w2 = 0.0;
        if (opt.nP > 0) {
            if (opt.nP % 4 != 0 || !ok(opt.nP, &w2)) return HTD_ERR_UNSTABLE;
            nP = opt.nP;
        } else {
            for (int q = 4; q < (1 << 20) && !nP; q += 4)
                if (ok(q, &w2)) nP = q;
            if (!nP) return HTD_ERR_UNSTABLE;
        }
        P.omega_c = std::sqrt(w2);
        P.lam_max_A = P.lam_max_reH + w2;
    } else if (opt.nP > 0) {
        const double sv = std::sin(kPi / opt.nP);
        if (opt.nP % 4 != 0 || !(sv * sv < ratio)) return HTD_ERR_UNSTABLE;
        nP = opt.nP;
    } else {
        for (int q = 4; q < (1 << 20) && !nP; q += 4) {
            const double sv = std::sin(kPi / q);
            if (sv * sv < ratio) nP = q;
        }
        if (!nP) return HTD_ERR_UNSTABLE;
    }
    P.nP = nP;
    P.T = opt.T;
    P.steps = (long long)opt.T * nP;
    P.dt = 2.0 * kPi / (P.omega_c * nP);
    const double x = P.omega_c * P.dt;
    P.alpha = x * x / (2.0 - 2.0 * std::cos(x));
    P.beta = x / std::sin(x);
    P.rho = (opt.rho > 0.0) ? opt.rho : 1.0 / opt.T;
    P.steps_per_launch = 0;
    P.tile[0] = P.tile[1] = P.tile[2] = 0;
    P.ctas_per_sm = 0;
    P.waves = 0;
    P.step_kernel = -1;
    P.rhs_per_cta = 0;
    return HTD_OK;
}

htd_status create_impl(const htd_grid *grid, const double *c_cell, const double *R_node,
                       double omega_phys, int bc, const htd_options *optp, htd_ctx *c)
{
    Plan pl;
    htd_status pst = plan_impl(grid, c_cell, R_node, omega_phys, bc, optp, &pl);
    if (pst != HTD_OK) return pst;
    const htd_options opt = pl.opt;
    const int d = pl.d;
    const int64_t N = pl.N;
    c->d = d;
    for (int a = 0; a < 3; ++a) c->n[a] = pl.n[a];
    for (int s = 0; s < 4; ++s) { c->S[s] = pl.S[s]; c->M[s] = pl.M[s]; }
    c->opt = opt;
    c->h = grid->h;
    c->omega_phys = omega_phys;
    c->m = opt.restart;
    c->kmin = pl.p.k_min;
    c->kmax = pl.p.k_max;
    c->omega = pl.p.omega_c;
    c->lam_reH = pl.p.lam_max_reH;
    c->lam_A = pl.p.lam_max_A;
    c->nP = pl.p.nP;
    c->T = pl.p.T;
    c->nsteps = pl.p.steps;
    c->dt = pl.p.dt;
    c->alpha = pl.p.alpha;
    c->beta = pl.p.beta;
    c->rho = pl.p.rho;
    const int nP = c->nP;
    HTD_CUDA(cudaGetDevice(&c->device));

    // ---- recurrence coefficients ------------------------------------------
    const double cK = c->dt * c->dt / c->alpha;          // dt^2 / alpha
    const double q = cK / (grid->h * grid->h);
    const double p = cK * c->omega * c->omega;
    c->C.c0 = 2.0 - p - q * std::ldexp(c->S[0], d);
    c->C.cs[0] = 0.0;
    for (int s = 1; s < 4; ++s) c->C.cs[s] = (s <= d) ? q * std::ldexp(c->S[s], d - s) : 0.0;
    for (int s = 0; s < 4; ++s) c->C.mt[s] = c->M[s];
    c->atab.resize(c->nsteps);
    c->btab.resize(c->nsteps);
    for (long long j = 0; j < c->nsteps; ++j) {
        const double chi = window_chi(1.0 - (double)j / (double)c->nsteps, c->rho);
        const double ph = 2.0 * kPi * (double)(j % nP) / nP;
        c->atab[j] = cK * chi * std::cos(ph);
        c->btab[j] = cK * chi * std::sin(ph);
    }

    // ---- layouts and device memory ----------------------------------------
    const bool mixed = opt.precision == HTD_MIXED;
    const bool abd = opt.integrator == HTD_ABD;
    const bool cell_damp = opt.damping == HTD_DAMP_CELL;
    c->esz = mixed ? sizeof(float) : sizeof(double);
    c->Lr = make_layout(d, c->n, c->esz);
    c->L64 = make_layout(d, c->n, sizeof(double));
    const Layout &L = c->Lr;
    const size_t bytes = c->esz * (size_t)L.total;
    c->rcap = opt.max_rhs;
    void **shared_arrs[] = {&c->kap, &c->dco};
    for (void **pp : shared_arrs) {
        HTD_CUDA(htd::dev_malloc(pp, bytes));
        HTD_CUDA(cudaMemset(*pp, 0, bytes));
    }
    void **rhs_arrs[] = {&c->fre, &c->fim, &c->u0, &c->u1};
    for (void **pp : rhs_arrs) {
        HTD_CUDA(htd::dev_malloc(pp, bytes * c->rcap));
        HTD_CUDA(cudaMemset(*pp, 0, bytes * c->rcap));
    }
    HTD_CUDA(htd::dev_malloc((void **)&c->err_dev, sizeof(int) * htd::kStatusWords));
    {
        int words[htd::kStatusWords] = {0, 0, 0, 0};
        const unsigned long long lim = (unsigned long long)opt.wait_limit_ns;
        std::memcpy(&words[2], &lim, sizeof(lim));
        HTD_CUDA(cudaMemcpy(c->err_dev, words, sizeof(words), cudaMemcpyHostToDevice));
    }
    HTD_CUDA(htd::dev_malloc((void **)&c->slot, sizeof(OutSlot) * c->rcap));
    HTD_CUDA(cudaMemset(c->slot, 0, sizeof(OutSlot) * c->rcap));
    if (opt.mode == HTD_MODE_PROJECT)
        HTD_CUDA(htd::dev_malloc(&c->acc, c->esz * 4 * (size_t)N * c->rcap));
    if (abd) {                                     // third state plane of I_abd
        HTD_CUDA(htd::dev_malloc(&c->u2, bytes * c->rcap));
        HTD_CUDA(cudaMemset(c->u2, 0, bytes * c->rcap));
    }
    HTD_CUDA(htd::dev_malloc((void **)&c->act_dev, sizeof(int) * (1 + c->rcap)));
    HTD_CUDA(cudaMemset(c->act_dev, 0, sizeof(int) * (1 + c->rcap)));
    c->Rs.act = c->act_dev;
    c->Rs.slots = c->rcap;
    c->Rs.stride = L.total;
    HTD_CUDA(htd::dev_malloc((void **)&c->kap64, sizeof(double) * c->L64.total));
    HTD_CUDA(htd::dev_malloc((void **)&c->imH, sizeof(double) * N));

    // per-cell kappa = (h omega_phys / c)^2 at the cell's stored position;
    // per-node d = 1 / (1 + L_ii / 2), L = (beta dt / alpha) Im H / omega
    std::vector<double> qk(L.total, 0.0), dc(L.total, 0.0), k64(c->L64.total, 0.0), imh(N);
    const int64_t nx = c->n[d - 1], ny = c->n[d - 2], nz = (d == 3) ? c->n[0] : 1;
    for (int64_t az = (d == 3 ? -1 : 0); az < (d == 3 ? nz : 1); ++az)
        for (int64_t ay = -1; ay < ny; ++ay)
            for (int64_t ax = -1; ax < nx; ++ax) {
                const int64_t ci = (d == 3) ? ((az + 1) * (ny + 1) + (ay + 1)) * (nx + 1) + (ax + 1)
                                            : (ay + 1) * (nx + 1) + (ax + 1);
                const double k = omega_phys / c_cell[ci];
                const double kap = (grid->h * k) * (grid->h * k);
                qk[L.node(ax, ay, az)] = q * kap;
                k64[c->L64.node(ax, ay, az)] = kap;
            }
    const double lcoef = c->beta * c->dt / c->alpha / c->omega;
    for (int64_t iz = 0; iz < nz; ++iz)
        for (int64_t iy = 0; iy < ny; ++iy)
            for (int64_t ix = 0; ix < nx; ++ix) {
                const int64_t ci = (iz * ny + iy) * nx + ix;
                const double ih = omega_phys * R_node[ci];
                imh[ci] = ih;
                // I_acd: d = 1 / (1 + L_ii/2); I_abd with node damping: the damping
                // coefficient beta dt omega_phys R_i / (alpha omega) (abd_step_kernel)
                dc[L.node(ix, iy, iz)] = abd ? lcoef * ih : 1.0 / (1.0 + 0.5 * lcoef * ih);
            }
    std::vector<double> rc64;                      // omega_phys R_cell (cell damping)
    if (cell_damp) {
        // R_cell = mean of R over the cell's grid corners; the coefficient goes to
        // the cell's stored position (like q kappa), Im H is assembled from it
        std::fill(dc.begin(), dc.end(), 0.0);
        std::fill(imh.begin(), imh.end(), 0.0);    // no diagonal part
        rc64.assign(c->L64.total, 0.0);
        for (int64_t az = (d == 3 ? -1 : 0); az < (d == 3 ? nz : 1); ++az)
            for (int64_t ay = -1; ay < ny; ++ay)
                for (int64_t ax = -1; ax < nx; ++ax) {
                    double sum = 0.0;
                    int cnt = 0;
                    for (int bz = 0; bz < (d == 3 ? 2 : 1); ++bz)
                        for (int by = 0; by < 2; ++by)
                            for (int bx = 0; bx < 2; ++bx) {
                                const int64_t x = ax + bx, y = ay + by, z = (d == 3) ? az + bz : 0;
                                if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz) continue;
                                sum += R_node[(z * ny + y) * nx + x];
                                ++cnt;
                            }
                    const double rcell = sum / cnt;
                    dc[L.node(ax, ay, az)] = lcoef * omega_phys * rcell;
                    rc64[c->L64.node(ax, ay, az)] = omega_phys * rcell;
                }
    }
    htd_status st = mixed ? upload_recurrence<float>(c, qk, dc) : upload_recurrence<double>(c, qk, dc);
    if (st != HTD_OK) return st;
    HTD_CUDA(cudaMemcpy(c->kap64, k64.data(), sizeof(double) * c->L64.total, cudaMemcpyHostToDevice));
    {
        double S2[4];
        for (int k = 0; k < 4; ++k) S2[k] = std::ldexp(c->S[k], d - k);
        HTD_CUDA(htd::dev_malloc((void **)&c->coefP, sizeof(double) * htd::h_planes(d) * (size_t)N));
        htd::launch_assemble_H(c->L64, c->kap64, S2, c->M, c->coefP, 0);
        HTD_CUDA(cudaGetLastError());
        if (cell_damp) {
            // Im H = sum_o M_s (sum of omega_phys R over the shared cells): the same
            // assembly with S = 0 and -M (coefficient 0 - (-M_s) * sum)
            double Z[4] = {0.0, 0.0, 0.0, 0.0}, Mn[4];
            for (int k = 0; k < 4; ++k) Mn[k] = -c->M[k];
            // coefI first: the handle owns it, so a failure below leaks nothing
            HTD_CUDA(htd::dev_malloc((void **)&c->coefI, sizeof(double) * htd::h_planes(d) * (size_t)N));
            double *rcell = nullptr;
            HTD_CUDA(htd::dev_malloc((void **)&rcell, sizeof(double) * c->L64.total));
            cudaError_t e = cudaMemcpy(rcell, rc64.data(), sizeof(double) * c->L64.total,
                                       cudaMemcpyHostToDevice);
            if (e == cudaSuccess) {
                htd::launch_assemble_H(c->L64, rcell, Z, Mn, c->coefI, 0);
                e = cudaDeviceSynchronize();
            }
            cudaFree(rcell);
            HTD_CUDA(e);
        }
    }
    HTD_CUDA(cudaMemcpy(c->imH, imh.data(), sizeof(double) * N, cudaMemcpyHostToDevice));

    // temporal blocking for the 2-D FP32 recurrence, picked by timing against the
    // one-step kernel, or as options.tblock asks (1: one step per launch, 4/8:
    // that depth); tb_rows and tb_form restrict the configurations tried
    {
        const int want = (opt.tblock == 1) ? 0 : opt.tblock;
        if (d == 2 && mixed && !abd && opt.tblock != 1) {
            htd_status ts = autotune_tb2d(c, want, opt.tb_rows);
            if (ts != HTD_OK) return ts;
        }
        // the plain FP64 2-D recurrence: one-step launches or the resident grid
        const bool fp64_res_form = opt.tb_form == HTD_TB_ANY || opt.tb_form == HTD_TB_RESIDENT;
        if (d == 2 && !mixed && !abd && opt.tblock == 0 && fp64_res_form) {
            htd_status ts = autotune_fp64_2d(c);
            if (ts != HTD_OK) return ts;
        }
    }

    // TMA-streamed 3-D FP32 step (HTD_S3_ZMARCH keeps the register z-march kernel)
    {
        if (d == 3 && mixed && !abd && opt.s3_kernel != HTD_S3_ZMARCH) {
            float *planes[6] = {(float *)c->u0, (float *)c->u1, (float *)c->kap, (float *)c->dco,
                                (float *)c->fre, (float *)c->fim};
            // option value -> kernel shape (0..2 one node per thread, kS3Pair pairs)
            c->s3_shape = (opt.s3_kernel == HTD_S3_PAIR) ? kS3Default : opt.s3_kernel - HTD_S3_NODE_32x8;
            if (c->s3_shape != kS3Pair && c->rcap > 1) c->s3_shape = kS3Pair;   // rhs batches
            if (c->s3_shape == kS3Pair) {
                c->use_s3 = htd::make_stream3d_pair_maps(L, planes, &c->s3maps, c->rcap);
                if (!c->use_s3) {                                  // odd layout: one node per thread
                    (void)cudaGetLastError();
                    c->s3_shape = 0;
                }
            }
            if (c->s3_shape != kS3Pair && c->rcap == 1)
                c->use_s3 = htd::make_stream3d_maps(L, c->s3_shape, planes, &c->s3maps);
            if (c->use_s3) {
                c->s3_stages = (opt.s3_stages == 0) ? 5 : opt.s3_stages;
                c->s3_rpc = 1;
                c->s3_zchunk = c->s3_shape == kS3Pair ? htd::stream3d_pair_zchunk(L, c->s3_stages)
                                                      : htd::stream3d_zchunk(L, c->s3_shape);
                // right-hand sides per CTA (pair kernel, handles with several rhs):
                // 2 when asked, or the faster of 1 and 2 timed with every rhs slot
                // active (each with its own z chunk)
                const bool multi = c->s3_shape == kS3Pair && c->rcap > 1;
                const int want_rpc = multi ? opt.s3_rhs_per_cta : 1;
                htd::RhsSet all = htd::RhsSet{};
                if (multi) {
                    std::vector<int> idx(c->rcap);
                    for (int k = 0; k < c->rcap; ++k) idx[k] = k;
                    htd::launch_set_act(c->act_dev, c->rcap, idx.data(), 0);
                    HTD_CUDA(cudaDeviceSynchronize());
                    all = c->Rs;
                }
                if (opt.s3_zchunk > 0) {
                    c->s3_zchunk = opt.s3_zchunk;
                    if (want_rpc == 2) {
                        c->s3_rpc = 2;
                        c->s3_stages = 4;
                    }
                } else if (want_rpc == 0) {
                    htd_status ts = autotune_s3_zchunk(c, all);
                    if (ts != HTD_OK) return ts;
                    const int z1 = c->s3_zchunk, st1 = c->s3_stages;
                    const float us1 = c->step_us;
                    c->s3_rpc = 2;
                    c->s3_stages = 4;
                    c->s3_zchunk = htd::stream3d_pair_zchunk(L, 4, 2);
                    if ((ts = autotune_s3_zchunk(c, all)) != HTD_OK) return ts;
                    if (!(c->step_us < us1)) {
                        c->s3_rpc = 1;
                        c->s3_stages = st1;
                        c->s3_zchunk = z1;
                        c->step_us = us1;
                    }
                } else {
                    if (want_rpc == 2) {
                        c->s3_rpc = 2;
                        c->s3_stages = 4;
                        c->s3_zchunk = htd::stream3d_pair_zchunk(L, 4, 2);
                    }
                    htd_status ts = autotune_s3_zchunk(c, all);
                    if (ts != HTD_OK) return ts;
                }
            }
            (void)cudaGetLastError();
        }
    }

    // Krylov workspace
    const size_t vb = sizeof(double2) * (size_t)N;
    HTD_CUDA(htd::dev_malloc((void **)&c->V, vb * (c->m + 1)));
    if (opt.krylov == HTD_FGMRES) HTD_CUDA(htd::dev_malloc((void **)&c->Z, vb * c->m));
    HTD_CUDA(htd::dev_malloc((void **)&c->w, vb));
    HTD_CUDA(htd::dev_malloc((void **)&c->t, vb));
    HTD_CUDA(htd::dev_malloc((void **)&c->r, vb));
    c->nb = htd::dots_blocks(N);
    HTD_CUDA(htd::dev_malloc((void **)&c->partial, sizeof(double2) * (size_t)c->nb * (kMaxRestart + 1)));
    HTD_CUDA(htd::dev_malloc((void **)&c->hdev, sizeof(double2) * 3 * 72));
    HTD_CUDA(htd::host_malloc((void **)&c->hhost, sizeof(double2) * 3 * 72));
    HTD_CUDA(cudaEventCreate(&c->pev[0]));
    HTD_CUDA(cudaEventCreate(&c->pev[1]));
    HTD_CUDA(cudaDeviceSynchronize());
    return HTD_OK;
}

}  // namespace

namespace htd {

void operator_view(const htd_ctx *c, OperatorView *out)
{
    out->L64 = c->L64;
    out->kap64 = c->kap64;
    out->coefP = c->coefP;
    out->coefI = c->coefI;
    out->imH = c->imH;
    for (int k = 0; k < 4; ++k) {
        out->S2[k] = std::ldexp(c->S[k], c->d - k);
        out->M[k] = c->M[k];
    }
    out->ih2 = 1.0 / (c->h * c->h);
    out->device = c->device;
}

void ctx_info(const htd_ctx *c, CtxInfo *out)
{
    out->N = c->Lr.N;
    out->m = c->m;
    out->rcap = c->rcap;
    out->runs = (c->opt.mode == HTD_MODE_EXACT) ? 2 : 1;
    out->krylov = c->opt.krylov;
    out->device = c->device;
    out->nsteps = c->nsteps;
}

htd_status ctx_stage_run(htd_ctx *c, int run, int n, const int *idx, const double2 *const *Fp,
                         double2 *const *Up, cudaStream_t s)
{
    if (n < 0 || n > c->rcap) return HTD_ERR_ARG;
    launch_set_act(c->act_dev, n, idx, s);
    if (n > 0) {
        if (c->opt.precision == HTD_MIXED)
            launch_split_batch<float>(c->Lr, Fp, (float *)c->fre, (float *)c->fim, c->Lr.total,
                                      run, c->act_dev, c->rcap, s);
        else
            launch_split_batch<double>(c->Lr, Fp, (double *)c->fre, (double *)c->fim, c->Lr.total,
                                       run, c->act_dev, c->rcap, s);
        launch_set_slots(c->slot, Up, run, (c->opt.mode == HTD_MODE_EXACT) ? 2 : 1, c->act_dev,
                         c->rcap, s);
    }
    HTD_CUDA(cudaGetLastError());
    return HTD_OK;
}

cudaGraph_t ctx_step_graph(htd_ctx *c)
{
    if (graphs_disabled(c)) return nullptr;
    if (c->opt.precision == HTD_MIXED) capture_steps<float>(c);
    else capture_steps<double>(c);
    return c->exec ? c->graph : nullptr;
}

htd_status ctx_run_steps(htd_ctx *c, cudaStream_t s)
{
    return (c->opt.precision == HTD_MIXED) ? run_steps<float>(c, s) : run_steps<double>(c, s);
}

void ctx_join_batch(htd_ctx *c)
{
    if (!c->use_res) return;
    c->use_res = false;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
    c->graph_tried = false;
    if (c->use_tb) c->step_us = c->tb.us_per_step;
}

void ctx_account(htd_ctx *c, int applies, long long steps)
{
    c->applies += applies;
    c->steps_run += steps;
}

void ctx_apply_H(htd_ctx *c, const double2 *X, const double2 *F, double2 *Y, cudaStream_t s)
{
    apply_H(c, X, F, Y, s);
}

void ctx_dots(htd_ctx *c, const double2 *V, int64_t ldv, int kcount, const double2 *w,
              double2 *out, cudaStream_t s)
{
    launch_dots(V, ldv, kcount, w, c->Lr.N, c->partial, c->nb, s);
    launch_reduce(c->partial, c->nb, kcount, out, s);
}

bool ctx_group_view(htd_ctx *c, CtxGroupView *out)
{
    if (c->d != 2 || c->opt.precision != HTD_MIXED || c->opt.integrator != HTD_ACD) return false;
    if (c->opt.launch & HTD_LAUNCH_NO_GROUP) return false;
    if (c->opt.mode != HTD_MODE_TABLE1 && c->opt.mode != HTD_MODE_EXACT) return false;
    if (!c->u2 || !c->u3) return false;
    out->L = c->Lr;
    out->u[0] = (float *)c->u0;
    out->u[1] = (float *)c->u1;
    out->u[2] = (float *)c->u2;
    out->u[3] = (float *)c->u3;
    out->kap = (const float *)c->kap;
    out->dco = (const float *)c->dco;
    out->fre = (const float *)c->fre;
    out->fim = (const float *)c->fim;
    out->C = cast_coef<float>(c->C);
    out->nsteps = c->nsteps;
    out->ab.resize(2 * (size_t)c->nsteps);
    for (long long j = 0; j < c->nsteps; ++j) {
        out->ab[j] = (float)c->atab[j];
        out->ab[c->nsteps + j] = (float)c->btab[j];
    }
    // the output steps of run_steps_direct (Table 1: snapshot a quarter period
    // before the end; both modes: the final state)
    out->jim = c->nsteps - c->nP / 4;
    out->jfin = c->nsteps;
    out->slot = c->slot;
    out->R = c->Rs;
    out->err = c->err_dev;
    out->rcap = c->rcap;
    return true;
}

htd_status ctx_zero_states(htd_ctx *c, cudaStream_t s)
{
    const size_t bytes = c->esz * (size_t)c->Lr.total * c->rcap;
    HTD_CUDA(cudaMemsetAsync(c->u0, 0, bytes, s));
    HTD_CUDA(cudaMemsetAsync(c->u1, 0, bytes, s));
    return HTD_OK;
}

htd_status ctx_take_error(htd_ctx *c)
{
    int flag = 0;
    HTD_CUDA(cudaMemcpy(&flag, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        HTD_CUDA(cudaMemset(c->err_dev, 0, sizeof(int)));
        return HTD_ERR_TIMEOUT;
    }
    return HTD_OK;
}

// ---- allocation (every device or pinned allocation of the library) --------

namespace {
std::atomic<long long> g_fail_after{-1};    // htd_test_fail_alloc: allocations left before a failure

bool fail_this_allocation()
{
    long long k = g_fail_after.load();
    while (k >= 0 && !g_fail_after.compare_exchange_weak(k, k - 1)) {
    }
    return k == 0;
}
}  // namespace

cudaError_t dev_malloc_raw(void **p, size_t bytes)
{
    if (fail_this_allocation()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t host_malloc_raw(void **p, size_t bytes)
{
    if (fail_this_allocation()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}

}  // namespace htd

extern "C" {

void htd_test_fail_alloc(long long after)
{
    htd::g_fail_after.store(after < 0 ? -1 : after);
}

htd_status htd_set_wait_limit(htd_handle h, long long limit_ns, int stall_test)
{
    if (!h || limit_ns < 0) return HTD_ERR_ARG;
    int words[3] = {stall_test ? 1 : 0, 0, 0};
    const unsigned long long lim = (unsigned long long)limit_ns;
    std::memcpy(&words[1], &lim, sizeof(lim));
    HTD_CUDA(cudaMemcpy(h->err_dev + 1, words, sizeof(words), cudaMemcpyHostToDevice));
    return HTD_OK;
}

void htd_default_options(htd_options *opt)
{
    if (!opt) return;
    opt->precision = HTD_FP64;
    opt->mode = HTD_MODE_TABLE1;
    opt->krylov = HTD_FGMRES;
    opt->T = 10;
    opt->rho = 0.25;
    opt->nP = 0;
    opt->stencil = HTD_STENCIL_Q1MIX;
    opt->restart = 20;
    opt->max_rhs = 1;
    opt->proj_periods = 1;
    opt->integrator = HTD_ACD;
    opt->damping = HTD_DAMP_NODE;
    opt->stencil_a = 0.5;
    opt->stencil_gamma = 1.0;
    opt->tblock = 0;
    opt->tb_rows = 0;
    opt->tb_form = HTD_TB_ANY;
    opt->s3_kernel = HTD_S3_PAIR;
    opt->s3_stages = 0;
    opt->s3_zchunk = 0;
    opt->s3_rhs_per_cta = 0;
    opt->launch = 0;
    opt->wait_limit_ns = 0;
}

htd_status htd_create(const htd_grid *grid, const double *c_cell_host, const double *R_node_host,
                      double omega_phys, int bc, const htd_options *opt, htd_handle *out)
{
    htd::NvtxRange nvtx_range("htd_create");
    if (!out) return HTD_ERR_ARG;
    htd_ctx *c = new (std::nothrow) htd_ctx();
    if (!c) return HTD_ERR_OOM;
    htd_status st = create_impl(grid, c_cell_host, R_node_host, omega_phys, bc, opt, c);
    if (st != HTD_OK) {
        free_ctx(c);
        return st;
    }
    *out = c;
    return HTD_OK;
}

htd_status htd_destroy(htd_handle h)
{
    if (!h) return HTD_OK;
    cudaDeviceSynchronize();
    free_ctx(h);
    return HTD_OK;
}

htd_status htd_plan(const htd_grid *grid, const double *c_cell_host, const double *R_node_host,
                    double omega_phys, int bc, const htd_options *opt, htd_params *out)
{
    if (!out) return HTD_ERR_ARG;
    Plan pl;
    htd_status st = plan_impl(grid, c_cell_host, R_node_host, omega_phys, bc, opt, &pl);
    if (st == HTD_OK) *out = pl.p;
    return st;
}

htd_status htd_get_params(htd_handle h, htd_params *out)
{
    if (!h || !out) return HTD_ERR_ARG;
    htd_params &P = *out;
    P.k_min = h->kmin;
    P.k_max = h->kmax;
    P.omega_c = h->omega;
    P.lam_max_reH = h->lam_reH;
    P.lam_max_A = h->lam_A;
    P.dt = h->dt;
    P.alpha = h->alpha;
    P.beta = h->beta;
    P.rho = h->rho;
    P.nP = h->nP;
    P.T = h->T;
    P.steps = h->nsteps;
    P.steps_per_launch = h->use_res ? (int)h->nsteps : h->use_tb ? h->tb.B : 1;
    P.tile[0] = h->use_res ? h->res.W : h->use_tb ? h->tb.TX : 0;
    P.tile[1] = h->use_res ? h->res.H : h->use_tb ? h->tb.TY : 0;
    P.tile[2] = h->use_res ? 2 : h->use_tb ? (h->tb.pair ? 2 : 1) : 0;
    P.ctas_per_sm = h->use_res ? 1 : h->use_tb ? h->tb.occ : 0;
    P.waves = h->use_res ? 1 : h->use_tb ? h->tb.waves : 0;
    if (h->use_s3) {
        static const int tx[4] = {32, 64, 128, 64}, ty[4] = {8, 4, 2, 8};
        const int sh = (h->s3_shape >= 0 && h->s3_shape < 4) ? h->s3_shape : 0;
        const Layout &L = h->Lr;
        P.tile[0] = tx[sh];
        P.tile[1] = ty[sh];
        P.tile[2] = h->s3_zchunk;
        P.ctas_per_sm = (sh == kS3Pair && h->s3_stages <= 5 && h->s3_rpc == 1) ? 3 : 2;
        int dev = 0, nsm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int64_t ctas = ((L.nx + tx[sh] - 1) / tx[sh]) * ((L.ny + ty[sh] - 1) / ty[sh]) *
                             ((L.nz + h->s3_zchunk - 1) / h->s3_zchunk);
        const int64_t slots = (int64_t)P.ctas_per_sm * nsm;
        P.waves = (int)((ctas + slots - 1) / slots);
    }
    P.step_kernel = (h->opt.integrator == HTD_ABD) ? 3
                    : h->use_res                    ? 4
                    : h->use_tb                     ? 1
                                                    : (h->use_s3 ? 2 : 0);
    P.rhs_per_cta = h->use_s3 ? h->s3_rpc : 1;
    return HTD_OK;
}

htd_status htd_apply_precond(htd_handle h, const void *F_dev, void *U_dev, void *stream)
{
    htd::NvtxRange nvtx_range("htd_apply_precond");
    if (!h || !F_dev || !U_dev || F_dev == U_dev) return HTD_ERR_ARG;
    return precond(h, (const double2 *)F_dev, (double2 *)U_dev, (cudaStream_t)stream);
}

htd_status htd_apply_H(htd_handle h, const void *X_dev, void *Y_dev, void *stream)
{
    if (!h || !X_dev || !Y_dev || X_dev == Y_dev) return HTD_ERR_ARG;
    apply_H(h, (const double2 *)X_dev, nullptr, (double2 *)Y_dev, (cudaStream_t)stream);
    HTD_CUDA(cudaGetLastError());
    return HTD_OK;
}

htd_status htd_residual_norm(htd_handle h, const void *F_dev, const void *U_dev, void *r_dev,
                             double *rel, void *stream)
{
    if (!h || !F_dev || !U_dev || !rel) return HTD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double2 *r = r_dev ? (double2 *)r_dev : h->r;
    apply_H(h, (const double2 *)U_dev, (const double2 *)F_dev, r, s);
    double rn, fn;
    htd_status st = norm(h, r, &rn, s);
    if (st != HTD_OK) return st;
    if ((st = norm(h, (const double2 *)F_dev, &fn, s)) != HTD_OK) return st;
    *rel = (fn > 0.0) ? rn / fn : 0.0;
    return HTD_OK;
}

htd_status htd_gmres_solve(htd_handle h, const void *F_dev, void *U_dev, double tol, int max_iters,
                           void *stream, htd_solve_info *info)
{
    htd::NvtxRange nvtx_range("htd_gmres_solve");
    if (!h || !F_dev || !U_dev || F_dev == U_dev || max_iters < 0) return HTD_ERR_ARG;
    return gmres(h, (const double2 *)F_dev, (double2 *)U_dev, tol, max_iters, (cudaStream_t)stream, info);
}

htd_status htd_gmres_solve_host(htd_handle h, const void *F_host, void *U_host, double tol,
                                int max_iters, void *stream, htd_solve_info *info)
{
    htd::NvtxRange nvtx_range("htd_gmres_solve_host");
    if (!h || !F_host || !U_host || max_iters < 0) return HTD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = sizeof(double2) * (size_t)h->Lr.N;
    if (!h->Fh) HTD_CUDA(htd::dev_malloc((void **)&h->Fh, vb));
    if (!h->Uh) HTD_CUDA(htd::dev_malloc((void **)&h->Uh, vb));
    HTD_CUDA(cudaMemcpyAsync(h->Fh, F_host, vb, cudaMemcpyHostToDevice, s));
    HTD_CUDA(cudaMemcpyAsync(h->Uh, U_host, vb, cudaMemcpyHostToDevice, s));
    htd_status st = gmres(h, h->Fh, h->Uh, tol, max_iters, s, info);
    if (st != HTD_OK && st != HTD_ERR_NOT_CONVERGED) return st;
    HTD_CUDA(cudaMemcpyAsync(U_host, h->Uh, vb, cudaMemcpyDeviceToHost, s));
    HTD_CUDA(cudaStreamSynchronize(s));
    return st;
}

htd_status htd_grad(htd_handle h, int nsrc, const void *F_dev, int nrec,
                    const int64_t *rec_idx_host, const void *d_dev, double tol, int max_iters,
                    void *grad_m_dev, void *grad_R_dev, double *misfit, void *stream,
                    htd_solve_info *info)
{
    htd::NvtxRange nvtx_range("htd_grad");
    if (!h || nsrc < 1 || !F_dev || nrec < 0 || !misfit || max_iters < 0 || !(tol > 0.0))
        return HTD_ERR_ARG;
    if (h->opt.damping != HTD_DAMP_NODE) return HTD_ERR_ARG;   // dH/dR is diagonal here
    if (nrec > 0 && (!rec_idx_host || !d_dev)) return HTD_ERR_ARG;
    const int64_t N = h->Lr.N;
    for (int k = 0; k < nrec; ++k)
        if (rec_idx_host[k] < 0 || rec_idx_host[k] >= N) return HTD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = sizeof(double2) * (size_t)N;
    if (!h->gU) HTD_CUDA(htd::dev_malloc((void **)&h->gU, vb));
    if (!h->gMu) HTD_CUDA(htd::dev_malloc((void **)&h->gMu, vb));
    if (!h->gR) HTD_CUDA(htd::dev_malloc((void **)&h->gR, vb));
    if (nrec > h->grec_cap) {
        if (h->gres) cudaFree(h->gres);
        if (h->grec) cudaFree(h->grec);
        h->gres = nullptr;
        h->grec = nullptr;
        h->grec_cap = 0;
        HTD_CUDA(htd::dev_malloc((void **)&h->gres, sizeof(double2) * nrec));
        HTD_CUDA(htd::dev_malloc((void **)&h->grec, sizeof(int64_t) * nrec));
        h->grec_cap = nrec;
    }
    if (nrec > 0)
        HTD_CUDA(cudaMemcpyAsync(h->grec, rec_idx_host, sizeof(int64_t) * nrec,
                                 cudaMemcpyHostToDevice, s));
    const bool want_grad = grad_m_dev || grad_R_dev;
    const int64_t ncell = (h->n[0] + 1) * (h->d >= 2 ? h->n[1] + 1 : 1) * (h->d == 3 ? h->n[2] + 1 : 1);
    if (grad_m_dev) HTD_CUDA(cudaMemsetAsync(grad_m_dev, 0, sizeof(double) * ncell, s));
    if (grad_R_dev) HTD_CUDA(cudaMemsetAsync(grad_R_dev, 0, sizeof(double) * N, s));
    htd_solve_info tot;
    std::memset(&tot, 0, sizeof(tot));
    tot.converged = 1;
    auto add = [&](const htd_solve_info &x) {
        tot.iterations += x.iterations;
        tot.restarts += x.restarts;
        tot.precond_applies += x.precond_applies;
        tot.steps += x.steps;
        tot.ms_total += x.ms_total;
        tot.ms_precond += x.ms_precond;
        tot.launches += x.launches;
        tot.rel_res_true = std::fmax(tot.rel_res_true, x.rel_res_true);
        tot.converged = tot.converged && x.converged;
    };
    std::vector<double2> res(nrec > 0 ? nrec : 1);
    double J = 0.0;
    htd_status st = HTD_OK;
    for (int src = 0; src < nsrc && st == HTD_OK; ++src) {
        const double2 *Fs = static_cast<const double2 *>(F_dev) + (size_t)src * N;
        htd_solve_info x;
        HTD_CUDA(cudaMemsetAsync(h->gU, 0, vb, s));
        st = gmres(h, Fs, h->gU, tol, max_iters, s, &x);
        add(x);
        if (st != HTD_OK) break;
        HTD_CUDA(cudaMemsetAsync(h->gR, 0, vb, s));
        if (nrec > 0) {
            htd::launch_receiver_residual(h->gU, static_cast<const double2 *>(d_dev) + (size_t)src * nrec,
                                          h->grec, nrec, h->gres, h->gR, s);
            HTD_CUDA(cudaGetLastError());
            HTD_CUDA(cudaMemcpyAsync(res.data(), h->gres, sizeof(double2) * nrec,
                                     cudaMemcpyDeviceToHost, s));
            HTD_CUDA(cudaStreamSynchronize(s));
            for (int k = 0; k < nrec; ++k) J += 0.5 * (res[k].x * res[k].x + res[k].y * res[k].y);
        }
        if (!want_grad) continue;
        HTD_CUDA(cudaMemsetAsync(h->gMu, 0, vb, s));
        st = gmres(h, h->gR, h->gMu, tol, max_iters, s, &x);
        add(x);
        if (st != HTD_OK) break;
        htd::launch_gradients(h->L64, h->M, h->omega_phys, h->gMu, h->gU,
                              static_cast<double *>(grad_m_dev), static_cast<double *>(grad_R_dev), s);
        HTD_CUDA(cudaGetLastError());
    }
    HTD_CUDA(cudaStreamSynchronize(s));
    if (!std::isfinite(J) && st == HTD_OK) st = HTD_ERR_NONFINITE;
    *misfit = J;
    if (info) *info = tot;
    return st;
}

htd_status htd_grad_td(htd_handle h, int nsrc, const void *F_dev, int nrec,
                       const int64_t *rec_idx_host, const void *d_dev, int checkpoint_every,
                       void *grad_m_dev, void *grad_R_dev, double *misfit, void *stream)
{
    htd::NvtxRange nvtx_range("htd_grad_td");
    if (!h || nsrc < 1 || !F_dev || nrec < 0 || !misfit || checkpoint_every < 0)
        return HTD_ERR_ARG;
    if (h->opt.mode != HTD_MODE_TABLE1 && h->opt.mode != HTD_MODE_EXACT) return HTD_ERR_ARG;
    if (h->opt.integrator != HTD_ACD) return HTD_ERR_ARG;    // the adjoint of I_acd only
    if (nrec > 0 && (!rec_idx_host || !d_dev)) return HTD_ERR_ARG;
    const int64_t N = h->Lr.N;
    for (int k = 0; k < nrec; ++k)
        if (rec_idx_host[k] < 0 || rec_idx_host[k] >= N) return HTD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (nrec > h->grec_cap) {
        if (h->gres) cudaFree(h->gres);
        if (h->grec) cudaFree(h->grec);
        h->gres = nullptr;
        h->grec = nullptr;
        h->grec_cap = 0;
        HTD_CUDA(htd::dev_malloc((void **)&h->gres, sizeof(double2) * nrec));
        HTD_CUDA(htd::dev_malloc((void **)&h->grec, sizeof(int64_t) * nrec));
        h->grec_cap = nrec;
    }
    if (nrec > 0)
        HTD_CUDA(cudaMemcpyAsync(h->grec, rec_idx_host, sizeof(int64_t) * nrec,
                                 cudaMemcpyHostToDevice, s));
    const int64_t ncell = (h->n[0] + 1) * (h->d >= 2 ? h->n[1] + 1 : 1) * (h->d == 3 ? h->n[2] + 1 : 1);
    if (grad_m_dev) HTD_CUDA(cudaMemsetAsync(grad_m_dev, 0, sizeof(double) * ncell, s));
    if (grad_R_dev) HTD_CUDA(cudaMemsetAsync(grad_R_dev, 0, sizeof(double) * N, s));
    const double2 *F = static_cast<const double2 *>(F_dev);
    const double2 *d = static_cast<const double2 *>(d_dev);
    double *gm = static_cast<double *>(grad_m_dev), *gR = static_cast<double *>(grad_R_dev);
    htd_status st = (h->opt.precision == HTD_MIXED)
                        ? grad_td_impl<float>(h, nsrc, F, nrec, d, checkpoint_every, gm, gR, misfit, s)
                        : grad_td_impl<double>(h, nsrc, F, nrec, d, checkpoint_every, gm, gR, misfit, s);
    if (st == HTD_OK) {
        int flag = 0;
        HTD_CUDA(cudaMemcpy(&flag, h->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) {
            cudaMemset(h->err_dev, 0, sizeof(int));
            st = HTD_ERR_TIMEOUT;
        }
    }
    return st;
}

const char *htd_status_string(htd_status s)
{
    switch (s) {
    case HTD_OK: return "ok";
    case HTD_ERR_ARG: return "invalid argument";
    case HTD_ERR_CUDA: return "CUDA runtime error";
    case HTD_ERR_OOM: return "device out of memory";
    case HTD_ERR_UNSTABLE: return "n_P violates the CFL bound or is not a multiple of 4";
    case HTD_ERR_NONFINITE: return "non-finite value";
    case HTD_ERR_NOT_CONVERGED: return "not converged within the iteration cap";
    case HTD_ERR_TIMEOUT: return "device-side wait timed out";
    case HTD_ERR_SIZE: return "problem larger than the fixed-size buffer of this call allows";
    }
    return "unknown status";
}

}  // extern "C"
