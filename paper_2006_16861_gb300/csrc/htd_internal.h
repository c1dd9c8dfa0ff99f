// Internal declarations shared by the libhtd translation units.
// Not part of the public ABI (include/htd.h is).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <cstdint>
#include <vector>

#include "htd.h"

namespace htd {

// Padded device layout of grid planes (recurrence state, forcing planes,
// per-node coefficients and per-cell coefficients share it).
//  - axes: 2-D (y, x), 3-D (z, y, x); x fastest.  Node (i0, i1[, i2]).
//  - node x index i_x is stored at column xl + i_x, so that node 0 of every
//    row sits on a 128-byte boundary; columns xl-1 and xl+nx are the zero
//    ghost ring; pitch is a multiple of 128 bytes.
//  - rows (and planes in 3-D) are shifted by one: row i_y + 1, plane i_z + 1;
//    rows 0 and ny+1 (planes 0 and nz+1) are ghosts.
//  - cell a (lower corner, a = -1..n-1 per axis) is stored exactly where the
//    node a would be: column xl + a_x, row a_y + 1, plane a_z + 1.  Node beta
//    then touches the cells stored at (row, col) - {0,1}^d.
struct Layout {
    int d;
    int64_t nx, ny, nz;     // nodes per axis (nz = 1 in 2-D)
    int64_t xl;             // column of node x = 0
    int64_t pitch;          // elements per row
    int64_t plane;          // elements per plane = pitch * (ny + 2)
    int64_t total;          // elements per padded array
    int64_t N;              // nx * ny * nz (compact node count)
    __host__ __device__ int64_t node(int64_t ix, int64_t iy, int64_t iz) const {
        return (iz + (d == 3 ? 1 : 0)) * plane + (iy + 1) * pitch + xl + ix;
    }
};

// Scalar coefficients of one recurrence step (precision T), see step kernels.
template <typename T>
struct StepCoef {
    T c0;       // 2 - p - q 2^d S_0
    T cs[4];    // q 2^{d-s} S_s for s >= 1
    T mt[4];    // M_s (mass weights per Hamming distance)
};

// Rounded arithmetic with no contraction left to the compiler, for float,
// double and float2 (paired FP32: each lane rounds like the scalar op), so
// that kernels evaluating the same expression on scalars or on node pairs
// produce bit-identical results.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// StepCoef as the operand type V of stencil2d (V = T, or float2 broadcasts)
template <typename V>
struct Stencil2dCoef {
    V c0, mt0, mt1, mt2, ncs1, ncs2;     // ncs = -cs
};

template <typename T>
__device__ __forceinline__ Stencil2dCoef<T> stencil2d_coef(const StepCoef<T> &C)
{
    return {C.c0, C.mt[0], C.mt[1], C.mt[2], -C.cs[1], -C.cs[2]};
}

__device__ __forceinline__ Stencil2dCoef<float2> stencil2d_coef2(const StepCoef<float> &C)
{
    auto b = [](float x) { return make_float2(x, x); };
    return {b(C.c0), b(C.mt[0]), b(C.mt[1]), b(C.mt[2]), b(-C.cs[1]), b(-C.cs[2])};
}

// (2 - K) u at one node of the 2-D cell-form operator (App. A), h^2-scaled
// coefficients as in StepCoef.  u<r><c>: u_j at row offset r, column offset c
// (m = -1, 0, p = +1); k<ay><ax>: q*kappa of the node's four cells; pm, p0, pp:
// u_{-1,-1} + u_{-1,+1}, u_{0,-1} + u_{0,+1}, u_{+1,-1} + u_{+1,+1}; hk0 = k00 + k01,
// hk1 = k10 + k11.  A shallow tree of independent partial sums (short
// dependency chains) with every rounding spelled out: the one-step kernel, the
// temporally blocked kernel and its node-pair form (V = float2) all give
// identical results.
template <typename V>
__device__ __forceinline__ V stencil2d(const Stencil2dCoef<V> &C, V umm, V um0, V ump, V u0m, V u00,
                                       V u0p, V upm, V up0, V upp, V k00, V k01, V k10, V k11,
                                       V pm, V p0, V pp, V hk0, V hk1)
{
    const V center = vfma(C.mt0, vadd(hk0, hk1), C.c0);
    const V edge = vadd(vadd(um0, up0), p0);
    const V corner = vadd(pm, pp);
    const V m1 = vadd(vfma(hk0, um0, vmul(hk1, up0)),
                      vfma(vadd(k00, k10), u0m, vmul(vadd(k01, k11), u0p)));
    const V m2 = vadd(vfma(k00, umm, vmul(k01, ump)), vfma(k10, upm, vmul(k11, upp)));
    const V r1 = vfma(center, u00, vmul(C.ncs1, edge));
    const V r2 = vfma(C.mt1, m1, vfma(C.mt2, m2, vmul(C.ncs2, corner)));
    return vadd(r1, r2);
}

// Output targets of a preconditioner run, read by the step kernels from device
// memory so that a captured graph can be replayed for any output vector.
struct OutSlot {
    double *final_part;   // &U[0].re or &U[0].im (stride 2 doubles), or null
    double *snap_part;    // &U[0].im (stride 2), or null
};

// Right-hand sides of one step launch.  The launch has `slots` rhs slots per
// tile; slot k processes rhs act[1 + k] when k < act[0] and returns at once
// otherwise.  The list lives in device memory, so one captured step sequence
// serves every subset of a batch (converged systems drop out without a new
// capture).  act == null: a single rhs, index 0, slot 0.  The per-rhs planes
// (u_j, u_{j-1}, Re F, Im F, the second state pair of the blocked kernel) lie
// `stride` elements apart; q*kappa and d are shared by all rhs; the output
// slot of rhs r is slot[r].
struct RhsSet {
    const int *act = nullptr;
    int slots = 1;
    int64_t stride = 0;
};

// rhs of slot k, false if the slot is idle
__device__ __forceinline__ bool rhs_of_slot(const RhsSet &R, int k, int &rhs)
{
    if (!R.act) {
        rhs = 0;
        return k == 0;
    }
    if (k >= __ldg(R.act)) return false;
    rhs = __ldg(R.act + 1 + k);
    return true;
}

// ---- tracing -------------------------------------------------------------------

// NVTX range for the scope (header-only NVTX3: a no-op unless a profiler that
// reads NVTX is attached, e.g. ncu --nvtx or Nsight Systems)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---- device allocation (htd_capi.cu) ---------------------------------------

// Every allocation the library makes goes through these: cudaMalloc /
// cudaMallocHost, unless the test hook htd_test_fail_alloc has armed a failure
// for this allocation (then cudaErrorMemoryAllocation, nothing allocated).
cudaError_t dev_malloc_raw(void **p, size_t bytes);
cudaError_t host_malloc_raw(void **p, size_t bytes);
template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes)
{
    return dev_malloc_raw(reinterpret_cast<void **>(p), bytes);
}
template <typename T>
cudaError_t host_malloc(T **p, size_t bytes)
{
    return host_malloc_raw(reinterpret_cast<void **>(p), bytes);
}

// Per-handle status words on the device (the `err` pointer the kernels get):
// err[0] error flag (a bounded wait gave up), err[1] stall test (the first
// neighbour wait of each CTA waits on a barrier nothing arrives on), err[2..3]
// the neighbour-wait bound in ns as one 64-bit word (0 = kDefaultWaitNs).
constexpr int kStatusWords = 4;
constexpr unsigned long long kDefaultWaitNs = 1000000000ull;

// ---- kernel launchers (htd_kernels.cu) --------------------------------------

// Number of kernels enqueued by this library (host counter, not thread-safe
// across handles used concurrently; used for statistics only).
extern long long g_launches;

// Launch through cudaLaunchKernelEx; with `overlap`, programmatic stream
// serialisation: the kernel may start while the previous kernel of the stream
// drains, and must call griddepcontrol.wait before it reads anything that
// kernel writes or writes anything that kernel reads.  Launch errors are left
// for cudaGetLastError.
template <typename... KArgs, typename... Args>
void launch_ex(void (*kern)(KArgs...), dim3 grd, unsigned threads, size_t smem, cudaStream_t s,
               bool overlap, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grd;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = overlap ? 1 : 0;
    (void)cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}

template <typename T>
void launch_step(const Layout &L, const T *u, T *um, const T *kap, const T *dco,
                 const T *fre, const T *fim, const StepCoef<T> &C, T a, T b,
                 const OutSlot *slot, int flags, cudaStream_t s, const RhsSet &R = RhsSet{});

template <typename T>
void launch_split(const Layout &L, const double2 *F, T *fre, T *fim, int flip, cudaStream_t s);

void launch_set_slot(OutSlot *slot, double *final_part, double *snap_part, cudaStream_t s);

// ---- backward-differences scheme (I_abd) ------------------------------------------

// u_{n+1} -> out from u = u_n, um = u_{n-1} (see abd_step_kernel); damp: per node
// (cell = false) or per cell (cell = true) damping coefficient plane
template <typename T>
void launch_abd_step(const Layout &L, const T *u, const T *um, T *out, const T *kap,
                     const T *damp, bool cell, const T *fre, const T *fim, const StepCoef<T> &C,
                     T a, T b, T cth, const OutSlot *slot, int flags, cudaStream_t s,
                     const RhsSet &R = RhsSet{});

// ---- projection read-out (mode HTD_MODE_PROJECT) ------------------------------

// acc (per rhs, astride apart; 4 planes of N in compact order: s_re, s_im,
// c_re, c_im) += (wc, ws) u with compensated (Kahan) additions; u padded
template <typename T>
void launch_project_accumulate(const Layout &L, const T *u, T *acc, int64_t astride, T wc, T ws,
                               const RhsSet &R, cudaStream_t s);
// U = scale (s - c) to each listed rhs's output slot (re -> final, im -> snap)
template <typename T>
void launch_project_finish(int64_t N, const T *acc, int64_t astride, double scale,
                           const OutSlot *slot, const RhsSet &R, cudaStream_t s);

// ---- right-hand-side batches --------------------------------------------------

constexpr int kMaxRhs = 256;     // rhs per handle (act list entries)

// act[0] = n, act[1 + k] = idx[k] (n <= kMaxRhs; the list travels as a kernel
// parameter, so the host array may be reused at once)
void launch_set_act(int *act, int n, const int *idx, cudaStream_t s);
// Re/Im planes of the listed rhs r: Fp[r] (device table of compact complex128
// vectors) -> fre/fim + r * stride
template <typename T>
void launch_split_batch(const Layout &L, const double2 *const *Fp, T *fre, T *fim, int64_t stride,
                        int flip, const int *act, int slots, cudaStream_t s);
// slot[r] of the listed rhs r -> parts of Up[r] (see set_slots_kernel)
void launch_set_slots(OutSlot *slot, double2 *const *Up, int run, int runs, const int *act,
                      int slots, cudaStream_t s);

// ---- handle internals used by the batch driver (htd_capi.cu) ------------------

struct CtxInfo {
    int64_t N;          // unknowns
    int m;              // restart length
    int rcap;           // rhs slots (max_rhs)
    int runs;           // real runs per application: 1 (Table 1) or 2 (EXACT)
    int krylov;         // HTD_FGMRES or HTD_LEFT_GMRES
    int device;
    long long nsteps;   // recurrence steps per run
};
void ctx_info(const htd_ctx *c, CtxInfo *out);
// stage run `run` of one application for the rhs idx[0..n) (n = 0: the
// handle's step kernels idle): active list, Re/Im planes from Fp[r], output
// slots into Up[r] (Fp, Up: device tables indexed by rhs)
htd_status ctx_stage_run(htd_ctx *c, int run, int n, const int *idx, const double2 *const *Fp,
                         double2 *const *Up, cudaStream_t s);
// the handle's captured step sequence (captured on first use), or null if
// graphs are off or the capture failed
cudaGraph_t ctx_step_graph(htd_ctx *c);
// the step sequence on a stream (graph launch or direct launches)
htd_status ctx_run_steps(htd_ctx *c, cudaStream_t s);
// A handle joining a batch leaves the resident-grid 2-D kernel (its one
// cooperative launch holds every SM, while a batch runs its handles side by
// side) for the blocked configuration tuned at create, and drops a graph
// captured with it.
void ctx_join_batch(htd_ctx *c);
// statistics of runs launched through a batch graph
void ctx_account(htd_ctx *c, int applies, long long steps);
// Y = H X or F - H X (FP64)
void ctx_apply_H(htd_ctx *c, const double2 *X, const double2 *F, double2 *Y, cudaStream_t s);
// out[k] = conj(V + k ldv) . w for k < kcount (device), through the handle's
// partial-sum buffer (kcount <= 65)
void ctx_dots(htd_ctx *c, const double2 *V, int64_t ldv, int kcount, const double2 *w,
              double2 *out, cudaStream_t s);
// read and clear the device error word: HTD_ERR_TIMEOUT if a bounded wait gave up
htd_status ctx_take_error(htd_ctx *c);

// What a group launch needs of a handle: false unless the handle is 2-D, FP32
// recurrence, I_acd, Table 1 or exact read-out, with the second state pair.
struct CtxGroupView {
    Layout L;
    float *u[4];
    const float *kap, *dco, *fre, *fim;
    StepCoef<float> C;
    std::vector<float> ab;       // a_j then b_j, as the blocked kernel rounds them
    long long nsteps, jim, jfin;
    const OutSlot *slot;
    RhsSet R;
    int *err;
    int rcap;
};
bool ctx_group_view(htd_ctx *c, CtxGroupView *out);
// zero the first state pair of every rhs slot (a run starts from rest)
htd_status ctx_zero_states(htd_ctx *c, cudaStream_t s);

// ---- temporally blocked 2-D recurrence (htd_tblock.cu) ------------------------

constexpr int kTbMaxSteps = 8;

// per-launch step data: forcing coefficients a_j, b_j of the nsub steps and
// their output flags (bit 0: snapshot, bit 1: final state)
template <typename T>
struct TbSteps {
    T a[kTbMaxSteps];
    T b[kTbMaxSteps];
    int flags[kTbMaxSteps];
    int nsub;
};

struct TbPlan {
    int B = 0;          // steps per launch (halo width)
    int RPT = 0;        // rows per thread
    int RG = 0;         // row groups: tile rows H = RG * RPT, threads 64 * RG (32 * RG
                        // for node pairs)
    bool pair = false;  // two adjacent columns per thread in paired FP32 instructions
    bool sd = false;    // (pair form) d staged in shared memory instead of registers
    int TX = 0, TY = 0; // owned tile
    int H = 0;          // tile rows including the halo
    size_t smem = 0;    // dynamic shared memory per CTA
    int grid_x = 0, grid_y = 0;
    int occ = 0;        // resident CTAs per SM
    int waves = 0;      // ceil(tiles / (SMs * occ))
    float us_per_step = 0.f;   // measured by the autotuner
};

// TMA descriptors of the planes u0, u1, u2, u3, q*kappa and d.
struct TbMaps {
    CUtensorMap m[6];
};

// The blocked-kernel configurations (B = 4 or 8 steps per launch, want_B = 0:
// both; rows per thread 8..20) that fit the device, for a 2-D grid.
template <typename T>
std::vector<TbPlan> tb2d_candidates(const Layout &L, int want_B);

// The four state planes are nrhs stacks of planes L.total elements apart (one
// per rhs, 3-D maps with the rhs as the outer coordinate); q*kappa is shared.
template <typename T>
bool make_tb2d_maps(const Layout &L, const TbPlan &p, T *const planes[6], TbMaps *maps,
                    int nrhs = 1);

// nsub <= B steps from the state pair (maps in0, in1) into the planes uC, uD;
// a timed-out TMA wait sets *err = 1.  overlap: the previous kernel on the
// stream is a blocked launch of the same sequence, so this launch may start
// while it drains (programmatic dependent launch): its prologue reads only
// q*kappa, d and the forcing, which no launch of the sequence writes, and it
// waits for the previous grid before it touches a state plane.
template <typename T>
void launch_tb2d(const TbPlan &p, const TbMaps &maps, int in0, int in1, const Layout &L, T *uC,
                 T *uD, const T *dco, const T *fre, const T *fim, const StepCoef<T> &C,
                 const TbSteps<T> &S, const OutSlot *slot, int *err, cudaStream_t s,
                 const RhsSet &R = RhsSet{}, bool overlap = false);

// ---- resident-grid 2-D step (htd_res2d.cu) ------------------------------------
//
// A whole run (all steps, one rhs, FP32 or FP64) in one cooperative launch:
// ntx x nty tiles of W x H nodes, one CTA per tile and at most one per SM,
// every tile's states, cells, d and forcing in shared memory; neighbouring
// tiles swap edge values through `xbuf` (xwords 64-bit words, zeroed by the
// launcher).
struct Res2dPlan {
    int W = 0, H = 0;            // tile (W even, at most 132); the last tile row / column may be smaller
    int ntx = 0, nty = 0;        // tiles (CTAs) per axis
    int rpt = 0;                 // interior rows per thread and strip (3, 5 or 8)
    int sw = 0;                  // row stride of the shared-memory arrays (72 or 136)
    size_t smem = 0;             // dynamic shared memory per CTA
    size_t xwords = 0;           // exchange buffer words
};

// Projection read-out inside the resident run: the new states of steps j >=
// j_acc are accumulated, with the compensated sums of the separate
// accumulation kernel, into acc (planes [s_re, s_im, c_re, c_im] of N compact
// nodes) with weights w[2k] = cos theta_k, w[2k+1] = -sin theta_k, k = (j + 1)
// mod nP.  j_acc >= nsteps: no accumulation.
template <typename T>
struct Res2dProj {
    int j_acc = 1 << 30;
    int nP = 1;
    const T *w = nullptr;
    T *acc = nullptr;
    int64_t N = 0;
};

// The plan for a 2-D grid in precision T, or false if the grid does not fit
// the SMs' shared memory at one tile per SM, or the device cannot launch
// cooperatively.
template <typename T>
bool res2d_plan(const Layout &L, Res2dPlan *p);
// Steps 0 .. nsteps-1 from zero states with forcing a_j Re F - b_j Im F
// (ab[2j] = a_j, ab[2j+1] = b_j); the new state of step jim - 1 goes to the
// snapshot output, that of step jfin - 1 to the final output (OutSlot of rhs
// 0).  A wait that runs out sets err[0] = 1.
template <typename T>
void launch_res2d(const Res2dPlan &p, const T *kap, const T *dco, const T *fre, const T *fim,
                  const Layout &L, const StepCoef<T> &C, const T *ab, int nsteps, int jim,
                  int jfin, const OutSlot *slot, unsigned long long *xbuf, int *err,
                  cudaStream_t s, const Res2dProj<T> &P = Res2dProj<T>{});

// ---- one persistent launch for many 2-D instances (htd_tblock.cu) -----------
//
// The blocked pair form of the 2-D step for a whole group of instances (each
// with its own size, coefficients, step count and right-hand-side slots) in
// one launch per run: a work queue of tasks (level k, instance, slot, tile),
// level k = steps k B .. k B + B - 1 of the instance's run, ordered by level;
// a tile starts level k when its 3 x 3 tile neighbourhood (same instance and
// slot) has finished level k - 1 (per-tile counters, release / acquire).

// one instance of a group (device memory; CUtensorMap carries the alignment
// the tensor maps need)
struct GroupInst {
    TbMaps maps;                 // u0, u1, u2, u3 (rhs stacks), q*kappa, d for the group's box
    float *u[4];                 // the state planes: pair (0, 1) and pair (2, 3)
    const float *dco, *fre, *fim;
    Layout L;
    StepCoef<float> C;
    const float *ab;             // a_j at [0, nsteps), b_j at [nsteps, 2 nsteps)
    long long nsteps, jim, jfin; // output steps: snapshot after step jim - 1, final after jfin - 1
    const OutSlot *slot;         // output slot per rhs
    RhsSet R;                    // active list, slots, per-rhs stride
    int *err;                    // the handle's status words
    int *done;                   // [slot][tile] levels completed in this run
    int grid_x, grid_y;
    int nlev;                    // levels per run, ceil(nsteps / B)
};

// queue of one run (device memory, except the counts)
struct GroupSched {
    const GroupInst *inst;       // sorted by nlev, largest first
    const long long *lev_off;    // [nlev_max + 1] first task of each level
    const long long *inst_off;   // [ninst + 1] first task of each instance within a level
    int ninst, nlev_max;
    long long ntasks;
    unsigned long long *head;    // next task (zeroed before each run)
    int *abort;                  // set when a wait gives up: no CTA takes another task
};

// The group plan (B = 8 steps, 8 rows per thread, 20 row groups, d staged:
// the pair configuration the tuner picks on large grids), or false if it does
// not fit the device.
bool group2d_plan(TbPlan *p);
// Persistent CTAs that fit the device at once for the group plan.
int group2d_ctas();
void launch_group2d(const TbPlan &p, const GroupSched &S, int ctas, cudaStream_t s);

// Assembled FP64 operator: coefficient planes (N doubles each) of the centre
// and of the positive offsets (the other half follows from symmetry):
// 14 planes in 3-D, 5 in 2-D, not yet scaled by 1/h^2.
__host__ __device__ constexpr int h_planes(int d) { return d == 3 ? 14 : 5; }
void launch_assemble_H(const Layout &L, const double *kap64, const double S2[4], const double M[4],
                       double *coefP, cudaStream_t s);
// Y = H X (F == null) or Y = F - H X, complex128 compact vectors.  Im H is the
// diagonal imH, plus the assembled planes coefI if given (cell damping).
void launch_apply_H(const Layout &L, const double *coefP, const double *imH, double ih2,
                    const double2 *X, const double2 *F, double2 *Y, cudaStream_t s,
                    const double *coefI = nullptr);

// partial[k * nb + b] = sum over block b of conj(V_k) w, k < kcount.
// dots_blocks: blocks per dot pass, 4 per SM of the current device (queried
// once per device), at most kMaxDotBlocks.
constexpr int kMaxDotBlocks = 1216;
int dots_blocks(int64_t N);
void launch_dots(const double2 *V, int64_t ldv, int kcount, const double2 *w, int64_t N,
                 double2 *partial, int nb, cudaStream_t s);
// out[k] = sum_b partial[k * nb + b] (fixed order)
void launch_reduce(const double2 *partial, int nb, int kcount, double2 *out, cudaStream_t s);
// w -= sum_k h[k] V_k  (h on the device)
void launch_sub_combination(const double2 *V, int64_t ldv, int kcount, const double2 *h,
                            double2 *w, int64_t N, cudaStream_t s);
// U += sum_k y[k] Z_k  (y on the device)
void launch_add_combination(const double2 *Z, int64_t ldz, int kcount, const double2 *y,
                            double2 *U, int64_t N, cudaStream_t s);
// v = w * scale (w == v allowed: scaled in place)
void launch_scale(const double2 *w, double scale, double2 *v, int64_t N, cudaStream_t s);

// ---- TMA-streamed 3-D step, FP32 (htd_stream3d.cu) -----------------------------

// TMA descriptors: u0, u1 and q*kappa with the x-y halo; d, Re F, Im F, u0, u1
// as exact node boxes.
struct Stream3Maps {
    CUtensorMap m[8];
};
// tile shape: 0 = 32 x 8 columns, 1 = 64 x 4, 2 = 128 x 2 (one node per thread)
bool make_stream3d_maps(const Layout &L, int shape, float *const planes[6], Stream3Maps *maps);
int stream3d_zchunk(const Layout &L, int shape);
// one step; from = 0: u_j in u0 and u_{j-1} (overwritten) in u1, from = 1 swapped
void launch_stream3d(const Stream3Maps &maps, int from, int shape, const Layout &L, float *um,
                     const StepCoef<float> &C, float a, float b, const OutSlot *slot, int flags,
                     int zchunk, int *err, cudaStream_t s);

// Same step with two x-adjacent nodes per thread in paired FP32 instructions
// (htd_stream3d_pair.cu): 64 x 8 column tiles, same maps layout (halo boxes
// 72 x 10).  Needs an even x lead and pitch.  The per-rhs planes (u0, u1,
// Re F, Im F) are nrhs stacks L.total elements apart (4-D maps, rhs
// outermost); q*kappa and d are shared.
bool make_stream3d_pair_maps(const Layout &L, float *const planes[6], Stream3Maps *maps,
                             int nrhs = 1);
// first z chunk to try for a ring of `stages` stages and `rpc` right-hand sides
// per CTA (3 CTAs per SM for rpc 1 with 4-5 stages, else 2)
int stream3d_pair_zchunk(const Layout &L, int stages, int rpc = 1);
size_t stream3d_pair_smem_bytes(int stages, int rpc = 1);
// overlap: the launch may start while the previous kernel of the stream drains
// (its prologue loads q*kappa, d and the forcing, which no step writes; the
// state planes are loaded after the wait for that kernel).  rpc: right-hand
// sides per CTA, 1 (any stages) or 2 (4 stages): a CTA then streams one column
// tile for two rhs slots, loading q*kappa and d once and computing each
// stencil coefficient once for both.
void launch_stream3d_pair(const Stream3Maps &maps, int from, const Layout &L, float *um,
                          const StepCoef<float> &C, float a, float b, const OutSlot *slot,
                          int flags, int zchunk, int stages, int *err, cudaStream_t s,
                          const RhsSet &R = RhsSet{}, bool overlap = false, int rpc = 1);

// Gradient through the recurrence (htd_grad_td): res = U[rec] - d and the
// adjoint forcing planes are/aim (padded, pre-zeroed) += Re/Im res at receivers
template <typename T>
void launch_residual_planes(const Layout &L, const double2 *U, const double2 *d,
                            const int64_t *rec, int nrec, double2 *res, T *are, T *aim,
                            cudaStream_t s);
// gm[cell] += cm sum lam_b M u_{k-1,g};  gR[node] += cR lam (u_k - u_{k-2})
template <typename T>
void launch_grad_td(const Layout &L, const double M[4], double cm, double cR, const T *lam,
                    const T *uk, const T *uk1, const T *uk2, double *gm, double *gR,
                    cudaStream_t s);

// Receiver residual res = U[rec] - d, and r[rec] += conj(res) (r pre-zeroed).
void launch_receiver_residual(const double2 *U, const double2 *d, const int64_t *rec, int nrec,
                              double2 *res, double2 *r, cudaStream_t s);
// gm[cell] += omega^2 Re sum_cell mu M U; gR[node] += omega Im(mu U) (either may be null)
void launch_gradients(const Layout &L, const double M[4], double omega_phys, const double2 *mu,
                      const double2 *U, double *gm, double *gR, cudaStream_t s);

// Read-only view of a handle's FP64 operator data (defined in htd_capi.cu).
struct OperatorView {
    Layout L64;             // layout of kap64 (compact N = L64.N)
    const double *kap64;    // (h k)^2 per cell
    const double *coefP;    // assembled operator (launch_assemble_H)
    const double *coefI;    // assembled non-diagonal Im H, or null
    const double *imH;      // omega_phys R per node
    double S2[4], M[4], ih2;
    int device;
};
void operator_view(const htd_ctx *c, OperatorView *out);

}  // namespace htd
