// Temporally blocked 2-D recurrence: B steps of I_acd (Def. of I_acd, with
// Table 1's windowed forcing) per launch from shared memory, tiles moved by TMA.
//
// Each CTA owns a TX x TY tile of nodes (TX = 64 - 2B) and needs it with a halo
// of B nodes (64 columns, H = TY + 2B rows), plus one more ring for the
// neighbour reads, and the q*kappa of the cells touching those nodes.  All
// three come from the padded device layout, where a cell sits at the position
// of its lower-corner node, so one TMA box of kBoxW x (H + 2) elements per
// array covers everything: one thread issues three cp.async.bulk.tensor copies
// (zero fill outside the array) that complete on one mbarrier; the box starts
// at a 16-byte aligned column.  The per-node d and the two forcing planes are
// read into registers (the pair form can stage d by a fourth box instead).  Consecutive launches of a step sequence overlap
// (programmatic dependent launch): a launch reads q*kappa, d and the forcing
// while the previous one drains and loads the state planes after it.
//
// Step s (s = 0 .. nsub-1) gives correct values on the ring-shrunk region
// R_s = [s+1, 63-s) x [s+1, H-s-1), whose stencil reads only R_{s-1}; after
// nsub <= B steps the owned core [B, B+TX) x [B, B+TY) holds u_{j+nsub} and
// u_{j+nsub-1}, which are stored to the other pair of global state planes (so
// that neighbouring CTAs never read a half-updated halo).  Every node of the
// tile is written in every step, without a per-node test: outside R_s the
// value is never read by a node of R_{s+1}, and outside the domain d = 0 (and
// the forcing is zero), so the update returns u_{j+s-1} = 0 there exactly and
// the zero Dirichlet ring stays zero.  Per node the arithmetic is exactly that of
// step2d_kernel (same expression, same order).
//
// Threads: 64 columns x RG row groups; a thread walks down its rows with a 3x3
// register window of u_j and a 2x2 window of cells.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "htd_internal.h"

namespace htd {

namespace {

constexpr int kW = 64;           // tile width including the halo
constexpr int kBoxW = 72;        // TMA box width: 64 + 2 pad columns + up to 3 for alignment, rounded
// threads = 64 columns x RG row groups (RG = 8 or 16)
constexpr unsigned long long kWaitLimitNs = kDefaultWaitNs;  // 1 s bound on the TMA-completion wait

template <typename T>
__host__ __device__ constexpr size_t tb2d_array_bytes(int H)
{
    return (((size_t)(H + 2) * kBoxW * sizeof(T)) + 127) & ~(size_t)127;
}

// `arrays` boxes (u_j, u_{j-1}, q*kappa and, for the pair form with d staged,
// d) and the mbarrier
template <typename T>
size_t tb2d_smem_bytes(int H, int arrays = 3)
{
    return arrays * tb2d_array_bytes<T>(H) + 16;
}

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// plain arrive (release at CTA scope: the arriving warp's shared-memory writes,
// ordered before it by __syncwarp, are visible to the thread whose wait completes)
__device__ __forceinline__ void mbar_arrive_cta(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// bounded wait on phase 0 of the mbarrier; false if the time limit ran out
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar)
{
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, 0)) {
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// state planes: (column, row, rhs)
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Programmatic dependent launch.  Code before grid_dep_wait() may run while
// the previous kernel of the stream drains (when the launch allows it); after
// it, everything that kernel wrote is visible.  grid_dep_launch() lets the
// next launch of the stream be scheduled onto SMs as this grid's CTAs retire.
// Both are no-ops for an ordinary launch.
__device__ __forceinline__ void grid_dep_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void grid_dep_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename T, int B, int RPT, int RG>
__global__ void __launch_bounds__(kW * RG, 1)
tb2d_kernel(const __grid_constant__ TbMaps maps, int in0, int in1, T *__restrict__ uC,
            T *__restrict__ uD, const T *__restrict__ dco, const T *__restrict__ fre,
            const T *__restrict__ fim, Layout L, StepCoef<T> C, TbSteps<T> S,
            const OutSlot *__restrict__ slot, int *__restrict__ err, RhsSet R)
{
    constexpr int W = kW, TX = W - 2 * B, BW = kBoxW;
    constexpr int H = RG * RPT, TY = H - 2 * B;
    constexpr int kAlign = 16 / (int)sizeof(T);          // TMA column alignment in elements
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int ae = (int)(tb2d_array_bytes<T>(H) / sizeof(T));   // elements per box slot
    T *smem_t = reinterpret_cast<T *>(smem_raw);
    T *su0 = smem_t;                                      // u_j   (box row r = stored row y0 + r)
    T *su1 = smem_t + ae;                                 // u_{j-1}
    T *sk = smem_t + 2 * ae;                              // q*kappa per cell
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_t + 3 * ae);

    const int tid = threadIdx.x;
    int rhs;
    if (!rhs_of_slot(R, (int)blockIdx.z, rhs)) return;
    // TMA destinations must be 128-byte aligned; refuse to run otherwise
    if (smem_u32(smem_raw) & 127u) {
        if (tid == 0) atomicExch(err, 1);
        return;
    }
    uC += rhs * R.stride;
    uD += rhs * R.stride;
    fre += rhs * R.stride;
    fim += rhs * R.stride;
    slot += rhs;
    const int64_t x0 = (int64_t)blockIdx.x * TX - B;      // global x of local column 0
    const int64_t y0 = (int64_t)blockIdx.y * TY - B;      // global y of local row 0
    // box origin: stored row y0 (local pad row 0 = global row y0 - 1), stored
    // column of local pad column 0 rounded down to the TMA alignment
    const int64_t c0 = L.xl + x0 - 1;
    const int xs = (int)(c0 - (c0 % kAlign));
    const int off = (int)(c0 - xs);                        // 0 .. kAlign-1

    // q*kappa, d and the forcing: no launch of the step sequence writes them, so
    // they are read before the wait for the previous launch
    const int ys = (int)y0;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, (unsigned)(3 * (size_t)(H + 2) * BW * sizeof(T)));
        tma_load_2d(sk, &maps.m[4], xs, ys, bar);
    }

    // this thread's nodes: column lx, rows row0 .. row0 + RPT - 1; their d and
    // forcing stay in registers for all the launch's steps
    const int lx = tid & (W - 1);
    const int row0 = (tid / W) * RPT;
    const int64_t gx = x0 + lx;
    const bool col_in_domain = gx >= 0 && gx < L.nx;
    T rd[RPT], rfr[RPT], rfi[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int64_t gy = y0 + row0 + i;
        const bool in = col_in_domain && gy >= 0 && gy < L.ny;
        const int64_t g = in ? (gy + 1) * L.pitch + L.xl + gx : 0;
        rd[i] = in ? dco[g] : T(0);
        rfr[i] = in ? fre[g] : T(0);
        rfi[i] = in ? fim[g] : T(0);
    }
    // per-step forcing coefficients and flags, staged in shared memory so that
    // the step loop does not index the parameter block dynamically
    __shared__ T s_a[kTbMaxSteps], s_b[kTbMaxSteps];
    __shared__ int s_flags[kTbMaxSteps];
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < kTbMaxSteps; ++q) {
            s_a[q] = S.a[q];
            s_b[q] = S.b[q];
            s_flags[q] = S.flags[q];
        }
    }

    grid_dep_wait();                                      // the state planes are final from here
    if (tid == 0) {
        tma_load_3d(su0, &maps.m[in0], xs, ys, rhs, bar);
        tma_load_3d(su1, &maps.m[in1], xs, ys, rhs, bar);
    }
    __syncthreads();                                      // barrier initialised before anyone waits
    const bool ok = mbar_wait_bounded(bar);
    if (__syncthreads_or(!ok)) {
        // give up: record it, wait (bounded) once more for the copies in flight, return
        if (tid == 0) {
            atomicExch(err, 1);
            mbar_wait_bounded(bar);
        }
        __syncthreads();
        return;
    }
    grid_dep_launch();

    // smem positions: node (ly, lx) at row ly + 1, column lx + 1 + off; its
    // cells (ly + ay, lx + ax) at row ly + ay, column lx + ax + off
    const bool col_owned = lx >= B && lx < B + TX;
    const int cc = lx + off;                               // smem column of (lx - 1)
    // rows of this tile inside the domain: y0 + ly in [0, ny)
    const int dom_lo = (int)max((int64_t)0, -y0);
    const int dom_hi = (int)min((int64_t)H, (int64_t)L.ny - y0);

    const Stencil2dCoef<T> SC = stencil2d_coef(C);

    // one step over this thread's rows; WITH_OUT: also write the owned nodes to
    // the output vector (the snapshot / final steps only)
    auto step = [&](int s, auto with_out) {
        constexpr bool kOut = decltype(with_out)::value;
        const T *__restrict__ cur = (s & 1) ? su1 : su0;   // u_{j+s}
        T *__restrict__ prv = (s & 1) ? su0 : su1;         // u_{j+s-1}, overwritten by u_{j+s+1}
        const T a = s_a[s], b = s_b[s];
        const int flags = s_flags[s];
        // window: rows row0 - 1 (m) and row0 (0); outer-pair sums of u rows and
        // horizontal sums of cell rows carried from row to row
        const T *cp = cur + row0 * BW + cc;
        T umm = cp[0], um0 = cp[1], ump = cp[2];
        T u0m = cp[BW], u00 = cp[BW + 1], u0p = cp[BW + 2];
        T pm = umm + ump, p0 = u0m + u0p;
        T k00 = sk[row0 * BW + cc], k01 = sk[row0 * BW + cc + 1];
        T hk0 = k00 + k01;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int ly = row0 + i;
            const T *np = cur + (ly + 2) * BW + cc;
            const T upm = np[0], up0 = np[1], upp = np[2];
            const T k10 = sk[(ly + 1) * BW + cc], k11 = sk[(ly + 1) * BW + cc + 1];
            const T pp = upm + upp;
            const T hk1 = k10 + k11;
            const T acc = stencil2d(SC, umm, um0, ump, u0m, u00, u0p, upm, up0, upp, k00, k01, k10,
                                    k11, pm, p0, pp, hk0, hk1);
            // every node stores (see the header: no per-node test is needed)
            const int ni = (ly + 1) * BW + cc + 1;
            const T ag = vfma(a, rfr[i], vfma(-b, rfi[i], acc));
            const T uprev = prv[ni];
            const T unew = vfma(rd[i], vfma(T(-2), uprev, ag), uprev);
            prv[ni] = unew;
            if (kOut && col_in_domain && col_owned && ly >= B && ly < B + TY && ly >= dom_lo &&
                ly < dom_hi) {
                const int64_t c = (y0 + ly) * L.nx + gx;
                if ((flags & 1) && slot->snap_part) slot->snap_part[2 * c] = (double)unew;
                if ((flags & 2) && slot->final_part) slot->final_part[2 * c] = (double)unew;
            }
            umm = u0m; um0 = u00; ump = u0p; pm = p0;
            u0m = upm; u00 = up0; u0p = upp; p0 = pp;
            k00 = k10; k01 = k11; hk0 = hk1;
        }
        __syncthreads();
    };
    for (int s = 0; s < S.nsub; ++s) {
        if (s_flags[s]) step(s, std::true_type{});
        else step(s, std::false_type{});
    }

    // ---- store the owned core of the last two states ----------------------
    const T *last = (S.nsub & 1) ? su1 : su0;               // u_{j+nsub}
    const T *prev = (S.nsub & 1) ? su0 : su1;               // u_{j+nsub-1}
    if (lx >= B && lx < B + TX && col_in_domain) {
        for (int ly = max(row0, B); ly < min(row0 + RPT, B + TY); ++ly) {
            const int64_t gy = y0 + ly;
            if (gy >= L.ny) break;
            const int64_t g = (gy + 1) * L.pitch + L.xl + gx;
            const int si = (ly + 1) * BW + cc + 1;
            uC[g] = last[si];
            uD[g] = prev[si];
        }
    }
}

// Node-pair form of tb2d_kernel (FP32): thread (p, g) owns the columns
// lx = 2p, 2p+1 of rows g RPT .. g RPT + RPT - 1, and every operation of the
// per-node update runs on the pair with the paired FP32 instructions (each
// lane rounds like the scalar instruction, so the results are those of
// tb2d_kernel and step2d_kernel).  The columns of a pair sit at an even shared
// memory column (the box starts one column left of a 16-byte boundary and
// tiles start at even x), so (lx, lx+1) is one 64-bit access; lx - 1 and
// lx + 2 are single loads.  SD: d comes from a fourth TMA box in shared memory
// (zero outside the domain, like the register copy) instead of registers,
// which frees 2 RPT registers per thread for more resident warps.
__device__ __forceinline__ float2 pr(float a, float b) { return make_float2(a, b); }

template <int B, int RPT, int RG, bool SD>
__global__ void __launch_bounds__(32 * RG, 1)
tb2d_pair_kernel(const __grid_constant__ TbMaps maps, int in0, int in1, float *__restrict__ uC,
                 float *__restrict__ uD, const float *__restrict__ dco,
                 const float *__restrict__ fre, const float *__restrict__ fim, Layout L,
                 StepCoef<float> C, TbSteps<float> S, const OutSlot *__restrict__ slot,
                 int *__restrict__ err, RhsSet R)
{
    typedef float T;
    constexpr int W = kW, TX = W - 2 * B, BW = kBoxW;
    constexpr int H = RG * RPT, TY = H - 2 * B;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int ae = (int)(tb2d_array_bytes<T>(H) / sizeof(T));
    T *smem_t = reinterpret_cast<T *>(smem_raw);
    T *su0 = smem_t;
    T *su1 = smem_t + ae;
    T *sk = smem_t + 2 * ae;
    T *sd = smem_t + 3 * ae;                               // SD only
    constexpr int kArrays = SD ? 4 : 3;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_t + kArrays * ae);

    const int tid = threadIdx.x;
    int rhs;
    if (!rhs_of_slot(R, (int)blockIdx.z, rhs)) return;
    const int64_t x0 = (int64_t)blockIdx.x * TX - B;
    const int64_t y0 = (int64_t)blockIdx.y * TY - B;
    const int64_t c0 = L.xl + x0 - 1;
    const int xs = (int)(c0 - (c0 % 4));
    const int off = (int)(c0 - xs);
    // TMA destinations 128-byte aligned and node pairs at even columns; refuse otherwise
    if ((smem_u32(smem_raw) & 127u) || !(off & 1)) {
        if (tid == 0) atomicExch(err, 1);
        return;
    }
    uC += rhs * R.stride;
    uD += rhs * R.stride;
    fre += rhs * R.stride;
    fim += rhs * R.stride;
    slot += rhs;

    // q*kappa, d and the forcing before the wait for the previous launch (as in
    // tb2d_kernel)
    const int ys = (int)y0;
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_expect_tx(bar, (unsigned)(kArrays * (size_t)(H + 2) * BW * sizeof(T)));
        tma_load_2d(sk, &maps.m[4], xs, ys, bar);
        if (SD) tma_load_2d(sd, &maps.m[5], xs, ys, bar);
    }

    const int lx = 2 * (tid & 31);                        // first column of the pair
    const int row0 = (tid >> 5) * RPT;
    const int64_t gx = x0 + lx;
    const bool inA = gx >= 0 && gx < L.nx, inB = gx + 1 >= 0 && gx + 1 < L.nx;
    float2 rd[SD ? 1 : RPT], rfr[RPT], rfi[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
        const int64_t gy = y0 + row0 + i;
        const bool rin = gy >= 0 && gy < L.ny;
        const int64_t g = rin ? (gy + 1) * L.pitch + L.xl + gx : 0;
        const bool a = rin && inA, b = rin && inB;
        if (!SD) rd[i] = pr(a ? dco[g] : 0.f, b ? dco[g + 1] : 0.f);
        rfr[i] = pr(a ? fre[g] : 0.f, b ? fre[g + 1] : 0.f);
        rfi[i] = pr(a ? fim[g] : 0.f, b ? fim[g + 1] : 0.f);
    }
    __shared__ T s_a[kTbMaxSteps], s_b[kTbMaxSteps];
    __shared__ int s_flags[kTbMaxSteps];
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < kTbMaxSteps; ++q) {
            s_a[q] = S.a[q];
            s_b[q] = S.b[q];
            s_flags[q] = S.flags[q];
        }
    }

    // Step-to-step order between row groups: warp g reads one halo row of its
    // neighbours g - 1 and g + 1 and overwrites rows they read one step earlier,
    // so before step s it waits only for those two to finish step s - 1 (one
    // mbarrier per warp and step parity, arrived on by the neighbours' lane 0),
    // instead of a barrier over the whole CTA.  Waits are bounded by the
    // handle's limit (err[2..3], read only when a wait does not complete at
    // once); a timeout sets *err and the abort word, and later waits are
    // skipped.  With the stall test (err[1]) warp 0's first wait is on `never`,
    // which nothing arrives on, so it runs out.
    __shared__ uint64_t nbar[2][RG];
    __shared__ uint64_t never;
    __shared__ int nabort, nstall;
    const int wg = tid >> 5, wl = tid & 31;
    if (tid == 0) {
        for (int q = 0; q < 2; ++q)
            for (int g = 0; g < RG; ++g)
                mbar_init(&nbar[q][g], (unsigned)((g > 0) + (g < RG - 1)));
        mbar_init(&never, 1u);
        nabort = 0;
        nstall = *(volatile const int *)(err + 1);
    }
    grid_dep_wait();
    if (tid == 0) {
        tma_load_3d(su0, &maps.m[in0], xs, ys, rhs, bar);
        tma_load_3d(su1, &maps.m[in1], xs, ys, rhs, bar);
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(bar);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            atomicExch(err, 1);
            mbar_wait_bounded(bar);
        }
        __syncthreads();
        return;
    }
    grid_dep_launch();

    const bool ownA = lx >= B && lx < B + TX;              // lx and lx+1 are owned together
    const int cc = lx + off;                               // smem column of lx - 1 (odd)
    const int dom_lo = (int)max((int64_t)0, -y0);
    const int dom_hi = (int)min((int64_t)H, (int64_t)L.ny - y0);
    const Stencil2dCoef<float2> SC = stencil2d_coef2(C);
    const float2 n2 = pr(-2.f, -2.f);

    // u row r of the plane as the pairs (m, 0, p) = (u(lx-1+o), u(lx+o)), o = 0, 1, 2
    auto urow = [&](const T *pl, int r, float2 &m, float2 &z, float2 &p) {
        const T *q = pl + r * BW + cc;
        const float l = q[0];
        z = *reinterpret_cast<const float2 *>(q + 1);
        const float rr = q[3];
        m = pr(l, z.x);
        p = pr(z.y, rr);
    };
    // cell row r: k0 = cells left of the nodes, k1 = cells right of them
    auto krow = [&](int r, float2 &k0, float2 &k1) {
        const T *q = sk + r * BW + cc;
        k1 = *reinterpret_cast<const float2 *>(q + 1);
        k0 = pr(q[0], k1.x);
    };

    auto step = [&](int s, auto with_out) {
        constexpr bool kOut = decltype(with_out)::value;
        const T *__restrict__ cur = (s & 1) ? su1 : su0;
        T *__restrict__ prv = (s & 1) ? su0 : su1;
        const float2 a2 = pr(s_a[s], s_a[s]), nb2 = pr(-s_b[s], -s_b[s]);
        const int flags = s_flags[s];
        float2 umm, um0, ump, u0m, u00, u0p;
        urow(cur, row0, umm, um0, ump);
        urow(cur, row0 + 1, u0m, u00, u0p);
        float2 pm = vadd(umm, ump), p0 = vadd(u0m, u0p);
        float2 k00, k01;
        krow(row0, k00, k01);
        float2 hk0 = vadd(k00, k01);
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int ly = row0 + i;
            float2 upm, up0, upp, k10, k11;
            urow(cur, ly + 2, upm, up0, upp);
            krow(ly + 1, k10, k11);
            const float2 pp = vadd(upm, upp);
            const float2 hk1 = vadd(k10, k11);
            const float2 acc = stencil2d(SC, umm, um0, ump, u0m, u00, u0p, upm, up0, upp, k00, k01,
                                         k10, k11, pm, p0, pp, hk0, hk1);
            const int ni = (ly + 1) * BW + cc + 1;
            const float2 ag = vfma(a2, rfr[i], vfma(nb2, rfi[i], acc));
            const float2 uprev = *reinterpret_cast<const float2 *>(prv + ni);
            const float2 dn = SD ? *reinterpret_cast<const float2 *>(sd + ni) : rd[SD ? 0 : i];
            const float2 unew = vfma(dn, vfma(n2, uprev, ag), uprev);
            *reinterpret_cast<float2 *>(prv + ni) = unew;   // no per-node test (header)
            if (kOut && ownA && ly >= B && ly < B + TY && ly >= dom_lo && ly < dom_hi) {
                const int64_t c = (y0 + ly) * L.nx + gx;
                if ((flags & 1) && slot->snap_part) {
                    if (inA) slot->snap_part[2 * c] = (double)unew.x;
                    if (inB) slot->snap_part[2 * c + 2] = (double)unew.y;
                }
                if ((flags & 2) && slot->final_part) {
                    if (inA) slot->final_part[2 * c] = (double)unew.x;
                    if (inB) slot->final_part[2 * c + 2] = (double)unew.y;
                }
            }
            umm = u0m; um0 = u00; ump = u0p; pm = p0;
            u0m = upm; u00 = up0; u0p = upp; p0 = pp;
            k00 = k10; k01 = k11; hk0 = hk1;
        }
    };
    const bool has_nb = RG > 1;
    for (int s = 0; s < S.nsub; ++s) {
        if (s > 0 && has_nb) {
            // the neighbours have finished step s - 1
            uint64_t *b = &nbar[(s - 1) & 1][wg];
            unsigned par = (unsigned)(((s - 1) >> 1) & 1);
            if (s == 1 && wg == 0 && nstall) {
                b = &never;
                par = 0;
            }
            if (!mbar_try_wait(b, par)) {
                const unsigned long long t0 = global_ns();
                unsigned long long lim =
                    *reinterpret_cast<volatile const unsigned long long *>(err + 2);
                if (lim == 0) lim = kDefaultWaitNs;
                while (!*(volatile int *)&nabort && !mbar_try_wait(b, par)) {
                    if (global_ns() - t0 > lim) {
                        *(volatile int *)&nabort = 1;
                        atomicExch(err, 1);
                    }
                }
            }
            __syncwarp();
        }
        if (s_flags[s]) step(s, std::true_type{});
        else step(s, std::false_type{});
        if (s + 1 < S.nsub && has_nb) {
            __syncwarp();                                // the warp's rows of step s written
            if (wl == 0) {
                if (wg > 0) mbar_arrive_cta(&nbar[s & 1][wg - 1]);
                if (wg < RG - 1) mbar_arrive_cta(&nbar[s & 1][wg + 1]);
            }
        }
    }
    __syncwarp();

    const T *last = (S.nsub & 1) ? su1 : su0;
    const T *prev = (S.nsub & 1) ? su0 : su1;
    if (ownA && (inA || inB)) {
        for (int ly = max(row0, B); ly < min(row0 + RPT, B + TY); ++ly) {
            const int64_t gy = y0 + ly;
            if (gy >= L.ny) break;
            const int64_t g = (gy + 1) * L.pitch + L.xl + gx;
            const int si = (ly + 1) * BW + cc + 1;
            if (inA) { uC[g] = last[si]; uD[g] = prev[si]; }
            if (inB) { uC[g + 1] = last[si + 1]; uD[g + 1] = prev[si + 1]; }
        }
    }
}

template <int B, int RPT, int RG, bool SD>
void add_pair_candidate(const Layout &L, std::vector<TbPlan> &out)
{
    constexpr int H = RG * RPT, TY = H - 2 * B, TX = kW - 2 * B, kThreads = 32 * RG;
    const size_t smem = tb2d_smem_bytes<float>(H, SD ? 4 : 3);
    if (H + 2 > 256 || smem > 220 * 1024) return;
    if (cudaFuncSetAttribute(tb2d_pair_kernel<B, RPT, RG, SD>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tb2d_pair_kernel<B, RPT, RG, SD>,
                                                      kThreads, smem) != cudaSuccess || occ < 1) {
        (void)cudaGetLastError();
        return;
    }
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    TbPlan p;
    p.B = B;
    p.RPT = RPT;
    p.RG = RG;
    p.pair = true;
    p.sd = SD;
    p.TX = TX;
    p.TY = TY;
    p.H = H;
    p.smem = smem;
    p.grid_x = (int)((L.nx + TX - 1) / TX);
    p.grid_y = (int)((L.ny + TY - 1) / TY);
    p.occ = occ;
    const int64_t slots = (int64_t)nsm * occ;
    p.waves = (int)(((int64_t)p.grid_x * p.grid_y + slots - 1) / slots);
    out.push_back(p);
}

template <typename T, int B, int RPT, int RG>
void add_candidate(const Layout &L, std::vector<TbPlan> &out)
{
    constexpr int H = RG * RPT, TY = H - 2 * B, TX = kW - 2 * B, kThreads = kW * RG;
    const size_t smem = tb2d_smem_bytes<T>(H);
    if (H + 2 > 256 || smem > 220 * 1024) return;
    if (cudaFuncSetAttribute(tb2d_kernel<T, B, RPT, RG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tb2d_kernel<T, B, RPT, RG>, kThreads, smem) !=
            cudaSuccess || occ < 1) {
        (void)cudaGetLastError();
        return;
    }
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    TbPlan p;
    p.B = B;
    p.RPT = RPT;
    p.RG = RG;
    p.TX = TX;
    p.TY = TY;
    p.H = H;
    p.smem = smem;
    p.grid_x = (int)((L.nx + TX - 1) / TX);
    p.grid_y = (int)((L.ny + TY - 1) / TY);
    p.occ = occ;
    const int64_t slots = (int64_t)nsm * occ;
    p.waves = (int)(((int64_t)p.grid_x * p.grid_y + slots - 1) / slots);
    out.push_back(p);
}

// ---- one persistent launch for a group of 2-D instances ---------------------

// queue offsets kept in shared memory up to these counts (global memory beyond)
constexpr int kGroupMaxLevels = 1024, kGroupMaxInst = 256;

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// orders this thread's generic-proxy view of global memory with its later (or
// earlier) bulk tensor copies
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent CTAs take tasks (level k, instance, rhs slot, tile) from a queue
// ordered by level.  A task is the work of one tb2d_pair_kernel CTA -- B steps
// of one tile from TMA-loaded shared memory, the same arithmetic in the same
// order, so the results are those of the per-instance launches bit for bit --
// started only when the 3 x 3 tiles around it (same instance and slot) have
// finished level k - 1: its halo then holds u_{kB}, u_{kB-1}, and no
// neighbour still reads the pair this task overwrites.  A task's dependencies
// have lower queue positions, so the lowest unfinished task can always run and
// the queue cannot deadlock (whatever number of CTAs is resident).  Every wait
// is bounded by the instance's limit; a wait that gives up sets the
// instance's error word and the group's abort word, and every CTA stops.
template <int B, int RPT, int RG, bool SD>
__global__ void __launch_bounds__(32 * RG, RG <= 8 ? 2 : 1)
tb2d_group_kernel(GroupSched Q)
{
    typedef float T;
    constexpr int W = kW, TX = W - 2 * B, BW = kBoxW;
    constexpr int H = RG * RPT, TY = H - 2 * B;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int ae = (int)(tb2d_array_bytes<T>(H) / sizeof(T));
    T *smem_t = reinterpret_cast<T *>(smem_raw);
    T *su0 = smem_t;
    T *su1 = smem_t + ae;
    T *sk = smem_t + 2 * ae;
    T *sd = smem_t + 3 * ae;                               // SD only
    constexpr int kArrays = SD ? 4 : 3;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_t + kArrays * ae);
    __shared__ T s_a[kTbMaxSteps], s_b[kTbMaxSteps];
    __shared__ int s_flags[kTbMaxSteps];
    __shared__ uint64_t nbar[2][RG];
    __shared__ int nabort, s_ok;
    __shared__ long long s_task, s_next;
    // the queue offsets, copied once per CTA (binary searches in shared memory)
    __shared__ long long s_lev[kGroupMaxLevels + 1], s_off[kGroupMaxInst + 1];
    __shared__ unsigned long long s_fenced;               // instances whose maps were acquired

    const int tid = threadIdx.x;
    const int wg = tid >> 5, wl = tid & 31;
    if (smem_u32(smem_raw) & 127u) {                      // TMA destinations 128-byte aligned
        if (tid == 0) atomicExch(Q.abort, 1);
        return;
    }
    const bool lev_in_smem = Q.nlev_max <= kGroupMaxLevels, off_in_smem = Q.ninst <= kGroupMaxInst;
    if (lev_in_smem)
        for (int i = tid; i <= Q.nlev_max; i += blockDim.x) s_lev[i] = Q.lev_off[i];
    if (off_in_smem)
        for (int i = tid; i <= Q.ninst; i += blockDim.x) s_off[i] = Q.inst_off[i];
    if (tid == 0) {
        s_fenced = 0ull;
        long long t = Q.ntasks;
        if (!*(volatile int *)Q.abort) t = (long long)atomicAdd(Q.head, 1ull);
        s_next = t;
    }
    const long long *lev_off = lev_in_smem ? s_lev : Q.lev_off;
    const long long *inst_off = off_in_smem ? s_off : Q.inst_off;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            // the task taken one round ahead; take the next one now, so that
            // the queue's latency is hidden behind this task
            const long long t = s_next;
            s_task = t;
            long long n = Q.ntasks;
            if (t < Q.ntasks && !*(volatile int *)Q.abort) n = (long long)atomicAdd(Q.head, 1ull);
            s_next = n;
        }
        __syncthreads();
        const long long task = s_task;
        if (task >= Q.ntasks) break;
        // level: the last k with lev_off[k] <= task; instance: the last i with
        // inst_off[i] <= task - lev_off[k] (instances sorted by level count,
        // so the ones still running at level k come first)
        int lo = 0, hi = Q.nlev_max;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (lev_off[mid] <= task) lo = mid; else hi = mid;
        }
        const int k = lo;
        const long long local = task - lev_off[k];
        lo = 0;
        hi = Q.ninst;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (inst_off[mid] <= local) lo = mid; else hi = mid;
        }
        const int inst = lo;
        const GroupInst &I = Q.inst[inst];
        const int ntile = I.grid_x * I.grid_y;
        const long long q = local - inst_off[inst];
        const int slot_k = (int)(q / ntile), tile = (int)(q % ntile);
        const int bx = tile % I.grid_x, by = tile / I.grid_x;
        int *done = I.done + (size_t)slot_k * ntile;
        int rhs;
        if (!rhs_of_slot(I.R, slot_k, rhs)) {             // idle slot: nothing to compute
            if (tid == 0) st_release_gpu(&done[tile], k + 1);
            continue;
        }
        const Layout &L = I.L;
        const int64_t x0 = (int64_t)bx * TX - B;
        const int64_t y0 = (int64_t)by * TY - B;
        const int64_t c0 = L.xl + x0 - 1;
        const int xs = (int)(c0 - (c0 % 4));
        const int off = (int)(c0 - xs);
        const int ys = (int)y0;
        const int rp = (k & 1) ? 2 : 0;                   // pair read at this level
        const int wp = 2 - rp;                            // pair written
        float *uC = I.u[wp] + rhs * I.R.stride;
        float *uD = I.u[wp + 1] + rhs * I.R.stride;
        const float *fre = I.fre + rhs * I.R.stride;
        const float *fim = I.fim + rhs * I.R.stride;
        const OutSlot *slot = I.slot + rhs;
        const long long j0 = (long long)k * B;
        const int nsub = (int)min((long long)B, I.nsteps - j0);

        if (wg == 0) {
            // the 3 x 3 tiles around have finished level k - 1: lane l < 9 polls
            // tile (l % 3 - 1, l / 3 - 1) (bounded wait; all nine at once)
            int ok = 1;
            if (k > 0) {
                const int nx_ = bx + (wl % 3) - 1, ny_ = by + (wl / 3) - 1;
                const bool mine = wl < 9 && nx_ >= 0 && ny_ >= 0 && nx_ < I.grid_x && ny_ < I.grid_y;
                const int *cnt = mine ? &done[ny_ * I.grid_x + nx_] : nullptr;
                unsigned long long lim = 0, t0 = 0;
                bool waited = false;
                for (;;) {
                    const bool ready = !mine || ld_acquire_gpu(cnt) >= k;
                    if (__all_sync(0xffffffffu, ready)) break;
                    if (!waited) {
                        waited = true;
                        t0 = global_ns();
                        lim = *reinterpret_cast<volatile const unsigned long long *>(I.err + 2);
                        if (lim == 0) lim = kDefaultWaitNs;
                    }
                    const bool give_up = *(volatile int *)Q.abort || global_ns() - t0 > lim;
                    if (__any_sync(0xffffffffu, give_up)) {
                        if (wl == 0) {
                            atomicExch(I.err, 1);
                            atomicExch(Q.abort, 1);
                        }
                        ok = 0;
                        break;
                    }
                }
                // lanes 1 .. 8 acquired their tiles' counters; the warp barrier
                // orders those acquires before lane 0's fence and copies
                __syncwarp();
                if (wl == 0) fence_proxy_async_global();   // the halo written by others, for TMA
            }
            // the steps' forcing coefficients and output flags, one lane each
            if (wl < kTbMaxSteps) {
                const long long j = j0 + wl;
                const bool in = wl < nsub;
                s_a[wl] = in ? I.ab[j] : 0.f;
                s_b[wl] = in ? I.ab[I.nsteps + j] : 0.f;
                int fl = 0;
                if (in && j + 1 == I.jim) fl |= 1;
                if (in && j + 1 == I.jfin) fl |= 2;
                s_flags[wl] = fl;
            }
            if (wl == 0) {
                s_ok = ok;
                nabort = 0;
                if (ok) {
                    // the tensor maps live in global memory (written by a host
                    // copy): acquired for the tensor-map proxy once per CTA and
                    // instance, before a copy uses them
                    const unsigned long long bit = (inst < 64) ? (1ull << inst) : 0ull;
                    if (!(s_fenced & bit)) {
                        for (int qq = 0; qq < 6; ++qq)
                            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                                             reinterpret_cast<uint64_t>(&I.maps.m[qq]))
                                         : "memory");
                        s_fenced |= bit;
                    }
                    mbar_init(bar, 1);
                    mbar_expect_tx(bar, (unsigned)(kArrays * (size_t)(H + 2) * BW * sizeof(T)));
                    tma_load_2d(sk, &I.maps.m[4], xs, ys, bar);
                    if (SD) tma_load_2d(sd, &I.maps.m[5], xs, ys, bar);
                    tma_load_3d(su0, &I.maps.m[rp], xs, ys, rhs, bar);
                    tma_load_3d(su1, &I.maps.m[rp + 1], xs, ys, rhs, bar);
                }
            }
        }
        // each warp initialises its own neighbour barriers (arrived on only
        // after the barrier below)
        if (wl == 0)
            for (int qq = 0; qq < 2; ++qq)
                mbar_init(&nbar[qq][wg], (unsigned)((wg > 0) + (wg < RG - 1)));
        __syncthreads();
        if (!s_ok) break;

        const int lx = 2 * wl;
        const int row0 = wg * RPT;
        const int64_t gx = x0 + lx;
        const bool inA = gx >= 0 && gx < L.nx, inB = gx + 1 >= 0 && gx + 1 < L.nx;
        float2 rd[SD ? 1 : RPT], rfr[RPT], rfi[RPT];
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int64_t gy = y0 + row0 + i;
            const bool rin = gy >= 0 && gy < L.ny;
            const int64_t g = rin ? (gy + 1) * L.pitch + L.xl + gx : 0;
            const bool a = rin && inA, b = rin && inB;
            if (!SD) rd[i] = pr(a ? I.dco[g] : 0.f, b ? I.dco[g + 1] : 0.f);
            rfr[i] = pr(a ? fre[g] : 0.f, b ? fre[g + 1] : 0.f);
            rfi[i] = pr(a ? fim[g] : 0.f, b ? fim[g + 1] : 0.f);
        }
        const bool ok = mbar_wait_bounded(bar);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(I.err, 1);
                atomicExch(Q.abort, 1);
                mbar_wait_bounded(bar);
            }
            __syncthreads();
            break;
        }

        const bool ownA = lx >= B && lx < B + TX;
        const int cc = lx + off;
        const int dom_lo = (int)max((int64_t)0, -y0);
        const int dom_hi = (int)min((int64_t)H, (int64_t)L.ny - y0);
        const Stencil2dCoef<float2> SC = stencil2d_coef2(I.C);
        const float2 n2 = pr(-2.f, -2.f);
        auto urow = [&](const T *pl, int r, float2 &m, float2 &z, float2 &p) {
            const T *qp = pl + r * BW + cc;
            const float l = qp[0];
            z = *reinterpret_cast<const float2 *>(qp + 1);
            const float rr = qp[3];
            m = pr(l, z.x);
            p = pr(z.y, rr);
        };
        auto krow = [&](int r, float2 &k0, float2 &k1) {
            const T *qp = sk + r * BW + cc;
            k1 = *reinterpret_cast<const float2 *>(qp + 1);
            k0 = pr(qp[0], k1.x);
        };
        auto step = [&](int s, auto with_out) {
            constexpr bool kOut = decltype(with_out)::value;
            const T *__restrict__ cur = (s & 1) ? su1 : su0;
            T *__restrict__ prv = (s & 1) ? su0 : su1;
            const float2 a2 = pr(s_a[s], s_a[s]), nb2 = pr(-s_b[s], -s_b[s]);
            const int flags = s_flags[s];
            float2 umm, um0, ump, u0m, u00, u0p;
            urow(cur, row0, umm, um0, ump);
            urow(cur, row0 + 1, u0m, u00, u0p);
            float2 pm = vadd(umm, ump), p0 = vadd(u0m, u0p);
            float2 k00, k01;
            krow(row0, k00, k01);
            float2 hk0 = vadd(k00, k01);
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int ly = row0 + i;
                float2 upm, up0, upp, k10, k11;
                urow(cur, ly + 2, upm, up0, upp);
                krow(ly + 1, k10, k11);
                const float2 pp = vadd(upm, upp);
                const float2 hk1 = vadd(k10, k11);
                const float2 acc = stencil2d(SC, umm, um0, ump, u0m, u00, u0p, upm, up0, upp, k00,
                                             k01, k10, k11, pm, p0, pp, hk0, hk1);
                const int ni = (ly + 1) * BW + cc + 1;
                const float2 ag = vfma(a2, rfr[i], vfma(nb2, rfi[i], acc));
                const float2 uprev = *reinterpret_cast<const float2 *>(prv + ni);
                const float2 dn = SD ? *reinterpret_cast<const float2 *>(sd + ni) : rd[SD ? 0 : i];
                const float2 unew = vfma(dn, vfma(n2, uprev, ag), uprev);
                *reinterpret_cast<float2 *>(prv + ni) = unew;
                if (kOut && ownA && ly >= B && ly < B + TY && ly >= dom_lo && ly < dom_hi) {
                    const int64_t c = (y0 + ly) * L.nx + gx;
                    if ((flags & 1) && slot->snap_part) {
                        if (inA) slot->snap_part[2 * c] = (double)unew.x;
                        if (inB) slot->snap_part[2 * c + 2] = (double)unew.y;
                    }
                    if ((flags & 2) && slot->final_part) {
                        if (inA) slot->final_part[2 * c] = (double)unew.x;
                        if (inB) slot->final_part[2 * c + 2] = (double)unew.y;
                    }
                }
                umm = u0m; um0 = u00; ump = u0p; pm = p0;
                u0m = upm; u00 = up0; u0p = upp; p0 = pp;
                k00 = k10; k01 = k11; hk0 = hk1;
            }
        };
        unsigned long long nlim = 0;
        for (int s = 0; s < nsub; ++s) {
            if (s > 0) {
                uint64_t *b = &nbar[(s - 1) & 1][wg];
                const unsigned par = (unsigned)(((s - 1) >> 1) & 1);
                if (!mbar_try_wait(b, par)) {
                    const unsigned long long t0 = global_ns();
                    if (nlim == 0) {
                        nlim = *reinterpret_cast<volatile const unsigned long long *>(I.err + 2);
                        if (nlim == 0) nlim = kDefaultWaitNs;
                    }
                    while (!*(volatile int *)&nabort && !mbar_try_wait(b, par)) {
                        if (global_ns() - t0 > nlim) {
                            *(volatile int *)&nabort = 1;
                            atomicExch(I.err, 1);
                            atomicExch(Q.abort, 1);
                        }
                    }
                }
                __syncwarp();
            }
            if (s_flags[s]) step(s, std::true_type{});
            else step(s, std::false_type{});
            if (s + 1 < nsub) {
                __syncwarp();
                if (wl == 0) {
                    if (wg > 0) mbar_arrive_cta(&nbar[s & 1][wg - 1]);
                    if (wg < RG - 1) mbar_arrive_cta(&nbar[s & 1][wg + 1]);
                }
            }
        }
        __syncwarp();
        // each warp stores its own rows of the owned core (reads of shared
        // memory only, so no barrier is needed before it)
        const T *last = (nsub & 1) ? su1 : su0;
        const T *prev = (nsub & 1) ? su0 : su1;
        if (ownA && (inA || inB)) {
            for (int ly = max(row0, B); ly < min(row0 + RPT, B + TY); ++ly) {
                const int64_t gy = y0 + ly;
                if (gy >= L.ny) break;
                const int64_t g = (gy + 1) * L.pitch + L.xl + gx;
                const int si = (ly + 1) * BW + cc + 1;
                if (inA) { uC[g] = last[si]; uD[g] = prev[si]; }
                if (inB) { uC[g + 1] = last[si + 1]; uD[g + 1] = prev[si + 1]; }
            }
        }
        __syncthreads();                                   // the core is stored by every thread
        if (tid == 0) {
            __threadfence();
            fence_proxy_async_global();
            st_release_gpu(&done[tile], k + 1);
            mbar_inval(bar);
        }
        if (wl == 0)
            for (int qq = 0; qq < 2; ++qq) mbar_inval(&nbar[qq][wg]);
    }
}

}  // namespace

template <typename T>
std::vector<TbPlan> tb2d_candidates(const Layout &L, int want_B)
{
    std::vector<TbPlan> v;
    if (L.d != 2) return v;
    if (want_B == 0 || want_B == 4) {
        add_candidate<T, 4, 12, 8>(L, v);
        add_candidate<T, 4, 20, 8>(L, v);
        add_candidate<T, 4, 6, 16>(L, v);
        add_candidate<T, 4, 10, 16>(L, v);
    }
    if (want_B == 0 || want_B == 8) {
        add_candidate<T, 8, 12, 8>(L, v);
        add_candidate<T, 8, 20, 8>(L, v);
        add_candidate<T, 8, 6, 16>(L, v);
        add_candidate<T, 8, 10, 16>(L, v);
    }
    if constexpr (std::is_same<T, float>::value) {
        if (want_B == 0 || want_B == 4) {
            add_pair_candidate<4, 10, 16, false>(L, v);
            add_pair_candidate<4, 6, 16, false>(L, v);
            add_pair_candidate<4, 12, 8, false>(L, v);
            add_pair_candidate<4, 8, 20, true>(L, v);
        }
        if (want_B == 0 || want_B == 8) {
            add_pair_candidate<8, 10, 16, false>(L, v);
            add_pair_candidate<8, 6, 16, false>(L, v);
            add_pair_candidate<8, 12, 8, false>(L, v);
            add_pair_candidate<8, 8, 20, true>(L, v);
            add_pair_candidate<8, 10, 16, true>(L, v);
        }
    }
    return v;
}

// Tensor maps of the planes u0, u1, u2, u3 (3-D: pitch x rows x nrhs), q*kappa
// and d (2-D: pitch x rows) with a kBoxW x (H + 2) box.
template <typename T>
bool make_tb2d_maps(const Layout &L, const TbPlan &p, T *const planes[6], TbMaps *maps, int nrhs)
{
    typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        (void)cudaGetLastError();
        return false;
    }
    EncodeFn encode = reinterpret_cast<EncodeFn>(fn);
    if (nrhs < 1) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)(L.ny + 2), (cuuint64_t)nrhs};
    const cuuint64_t strides[2] = {(cuuint64_t)(L.pitch * sizeof(T)),
                                   (cuuint64_t)(L.total * sizeof(T))};
    const cuuint32_t box[3] = {(cuuint32_t)kBoxW, (cuuint32_t)(p.H + 2), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    for (int i = 0; i < 6; ++i) {
        const cuuint32_t rank = (i < 4) ? 3 : 2;
        if (encode(&maps->m[i], dt, rank, (void *)planes[i], dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return false;
    }
    return true;
}

template <typename T>
void launch_tb2d(const TbPlan &p, const TbMaps &maps, int in0, int in1, const Layout &L, T *uC,
                 T *uD, const T *dco, const T *fre, const T *fim, const StepCoef<T> &C,
                 const TbSteps<T> &S, const OutSlot *slot, int *err, cudaStream_t s,
                 const RhsSet &R, bool overlap)
{
    dim3 grd((unsigned)p.grid_x, (unsigned)p.grid_y, (unsigned)R.slots);
    if constexpr (std::is_same<T, float>::value) {
#define HTD_TB2D_PAIR_CASE(BB, RR, GG, SS)                                                      \
        if (p.pair && p.B == BB && p.RPT == RR && p.RG == GG && p.sd == SS) {                   \
            launch_ex(tb2d_pair_kernel<BB, RR, GG, SS>, grd, 32 * GG, p.smem, s, overlap, maps,  \
                      in0, in1, uC, uD, dco, fre, fim, L, C, S, slot, err, R);                  \
            ++g_launches;                                                                       \
            return;                                                                             \
        }
        HTD_TB2D_PAIR_CASE(4, 10, 16, false)
        HTD_TB2D_PAIR_CASE(4, 6, 16, false)
        HTD_TB2D_PAIR_CASE(4, 12, 8, false)
        HTD_TB2D_PAIR_CASE(4, 8, 20, true)
        HTD_TB2D_PAIR_CASE(8, 10, 16, false)
        HTD_TB2D_PAIR_CASE(8, 6, 16, false)
        HTD_TB2D_PAIR_CASE(8, 12, 8, false)
        HTD_TB2D_PAIR_CASE(8, 8, 20, true)
        HTD_TB2D_PAIR_CASE(8, 10, 16, true)
#undef HTD_TB2D_PAIR_CASE
    }
    if (p.pair) return;
#define HTD_TB2D_CASE(BB, RR, GG)                                                              \
    if (p.B == BB && p.RPT == RR && p.RG == GG) {                                              \
        launch_ex(tb2d_kernel<T, BB, RR, GG>, grd, kW * GG, p.smem, s, overlap, maps, in0, in1,   \
                  uC, uD, dco, fre, fim, L, C, S, slot, err, R);                               \
        ++g_launches;                                                                          \
        return;                                                                                \
    }
    HTD_TB2D_CASE(4, 12, 8)
    HTD_TB2D_CASE(4, 20, 8)
    HTD_TB2D_CASE(4, 6, 16)
    HTD_TB2D_CASE(4, 10, 16)
    HTD_TB2D_CASE(8, 12, 8)
    HTD_TB2D_CASE(8, 20, 8)
    HTD_TB2D_CASE(8, 6, 16)
    HTD_TB2D_CASE(8, 10, 16)
#undef HTD_TB2D_CASE
}

// The group plan: node pairs, 8 steps per task, 8 rows per thread, 20 row
// groups, d staged in shared memory (the configuration the tuner picks on the
// large 2-D grids; one CTA per SM).  Measured against it on the batched
// workload's 64 instances: 4 steps per task on 56 x 152 tiles (1.37 times the
// useful nodes computed instead of 1.67) took 25 % longer, and 4 steps, 10
// rows, 8 groups with two CTAs per SM 22 % longer: the fixed cost of a task
// (its tile's copies in and out, the neighbour check) outweighs the halo.
constexpr int kGB = 8, kGRPT = 8, kGRG = 20;
constexpr bool kGSD = true;

bool group2d_plan(TbPlan *p)
{
    constexpr int H = kGRG * kGRPT;
    const size_t smem = tb2d_smem_bytes<float>(H, kGSD ? 4 : 3);
    if (cudaFuncSetAttribute(tb2d_group_kernel<kGB, kGRPT, kGRG, kGSD>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    p->B = kGB;
    p->RPT = kGRPT;
    p->RG = kGRG;
    p->pair = true;
    p->sd = kGSD;
    p->TX = kW - 2 * kGB;
    p->TY = H - 2 * kGB;
    p->H = H;
    p->smem = smem;
    p->grid_x = p->grid_y = 0;
    p->occ = 0;
    p->waves = 0;
    return group2d_ctas() > 0;
}

int group2d_ctas()
{
    constexpr int H = kGRG * kGRPT;
    const size_t smem = tb2d_smem_bytes<float>(H, kGSD ? 4 : 3);
    int occ = 0, dev = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tb2d_group_kernel<kGB, kGRPT, kGRG, kGSD>,
                                                      32 * kGRG, smem) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return occ * nsm;
}

void launch_group2d(const TbPlan &p, const GroupSched &S, int ctas, cudaStream_t s)
{
    tb2d_group_kernel<kGB, kGRPT, kGRG, kGSD><<<ctas, 32 * kGRG, p.smem, s>>>(S);
    ++g_launches;
}

template std::vector<TbPlan> tb2d_candidates<float>(const Layout &, int);
template bool make_tb2d_maps<float>(const Layout &, const TbPlan &, float *const[6], TbMaps *, int);
template void launch_tb2d<float>(const TbPlan &, const TbMaps &, int, int, const Layout &, float *,
                                 float *, const float *, const float *, const float *,
                                 const StepCoef<float> &, const TbSteps<float> &, const OutSlot *,
                                 int *, cudaStream_t, const RhsSet &, bool);

}  // namespace htd
