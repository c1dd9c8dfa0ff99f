// 3-D recurrence step streamed by TMA, two x-adjacent nodes per thread (FP32).
//
// Same method and pipeline as stream3d_kernel (one step of I_acd with Table 1's
// windowed forcing; a producer warp streams z planes of a column tile through
// a ring of shared-memory stages with full/empty mbarriers; consumer warps keep
// register windows over three planes), but each consumer thread updates the
// pair of nodes (x, x+1), x = x0 + 2 tx, so that the 27-term stencil sum, the
// cell sums of q*kappa and the update run on float2 pairs with the paired FP32
// instructions of sm_100+ (__ffma2_rn, __fadd2_rn, __fmul2_rn): about half the
// FP instructions and half the per-node bookkeeping of the one-node kernel.
//
// Tile: 64 x 8 columns (256 consumer threads).  Stage = u_j box and q*kappa box
// (72 x 10: columns x0-1 .. x0+64 with the 16-byte aligned start, rows
// y0-1 .. y0+8) and exact 64 x 8 boxes of d, Re F, Im F, u_{j-1}.  In the halo
// boxes node column x sits at box column x - x0 + 1 + off with off = 3 (the
// padded layout puts column x0 - 1 at 3 mod 4), so (x, x+1) for even x - x0
// is an aligned 64-bit pair and x - 1, x + 2 are single loads.  The two halo
// planes of a z chunk (below and above its node planes) load only u_j, plus
// q*kappa for the lower one: their node boxes would never be read, and as the
// neighbouring chunk runs in another wave they would come from DRAM.
//
// Per node the arithmetic is the one-node kernel's, in the same order, with
// each scalar operation replaced by the same operation on a pair; paired
// instructions round each lane exactly like the scalar ones.
#include <cuda.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "htd_internal.h"

namespace htd {

namespace {

constexpr int kTX = 64, kTY = 8;
constexpr int kThreads = 256;                   // consumer threads, 2 nodes each
constexpr int kHaloW = 72, kHaloH = kTY + 2;
constexpr int kHaloElems = kHaloW * kHaloH;     // 720 floats copied
constexpr int kHaloStride = 768;                // padded to 3072 bytes (128-byte multiple)
constexpr int kNodeElems = kTX * kTY;           // 512 floats
// Stage layout for RPC right-hand sides per CTA: the u_j halo box of each rhs,
// the q*kappa halo box, d, then Re F, Im F, u_{j-1} of each rhs.  RPC = 1 is the
// single-rhs layout [u_j | q*kappa | d | Re F | Im F | u_{j-1}].
template <int RPC>
__host__ __device__ constexpr int stage_elems()
{
    return (RPC + 1) * kHaloStride + (1 + 3 * RPC) * kNodeElems;
}
// bytes a stage's copies bring: node planes of the chunk (everything) and the
// two halo planes (u_j and q*kappa on the lower one, u_j on the upper one),
// for `nr` right-hand sides present in the CTA
__host__ __device__ constexpr unsigned stage_tx_bytes(int kind, int nr)
{
    return kind == 0 ? (unsigned)(((nr + 1) * kHaloElems + (1 + 3 * nr) * kNodeElems) * 4)
         : kind == 1 ? (unsigned)((nr + 1) * kHaloElems * 4)
                     : (unsigned)(nr * kHaloElems * 4);
}
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

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

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool wait_bounded(uint64_t *bar, unsigned phase, volatile int *abort_flag)
{
    if (mbar_try_wait(bar, phase)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, phase)) {
        if (*abort_flag) return false;
        if (global_ns() - t0 > kWaitLimitNs) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// per-rhs planes: (column, row, plane, rhs)
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            int r, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(r), "r"(smem_u32(bar))
        : "memory");
}

// Stored plane p into one stage for the rhs r[0 .. nr) of the CTA: u_j and
// q*kappa with the halo, d, Re F, Im F, u_{j-1}.  The stage's byte count is
// announced first; the coefficient part (q*kappa, d, forcing: no step writes
// them) and the state part (u_j, u_{j-1}) may be issued separately.  `kind` 0:
// a node plane of the chunk (everything); 1: the lower halo plane (u_j,
// q*kappa); 2: the upper halo plane (u_j only).  The node boxes of a halo
// plane are never read.
template <int RPC>
__device__ __forceinline__ void load_stage_coef(const Stream3Maps &maps, float *stage, uint64_t *bar,
                                                int xs, int xn, int y0, int p, const int *r, int nr,
                                                int kind)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(stage_tx_bytes(kind, nr))
                 : "memory");
    if (kind == 2) return;
    tma_load_3d(stage + RPC * kHaloStride, &maps.m[2], xs, y0, p, bar);
    if (kind == 1) return;
    float *nd = stage + (RPC + 1) * kHaloStride;
    tma_load_3d(nd, &maps.m[3], xn, y0 + 1, p, bar);
    for (int q = 0; q < nr; ++q) {
        float *nq = nd + kNodeElems + q * 3 * kNodeElems;
        tma_load_4d(nq, &maps.m[4], xn, y0 + 1, p, r[q], bar);
        tma_load_4d(nq + kNodeElems, &maps.m[5], xn, y0 + 1, p, r[q], bar);
    }
}

template <int RPC>
__device__ __forceinline__ void load_stage_state(const Stream3Maps &maps, int iu, int ium,
                                                 float *stage, uint64_t *bar, int xs, int xn,
                                                 int y0, int p, const int *r, int nr, int kind)
{
    float *nd = stage + (RPC + 1) * kHaloStride;
    for (int q = 0; q < nr; ++q) {
        tma_load_4d(stage + q * kHaloStride, &maps.m[iu], xs, y0, p, r[q], bar);
        if (kind == 0)
            tma_load_4d(nd + kNodeElems + q * 3 * kNodeElems + 2 * kNodeElems, &maps.m[ium], xn,
                        y0 + 1, p, r[q], bar);
    }
}

// programmatic dependent launch (no-ops for an ordinary launch): code before
// grid_dep_wait() may overlap the previous kernel of the stream; after it,
// everything that kernel wrote is visible
__device__ __forceinline__ void grid_dep_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ void grid_dep_launch()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// pair helpers
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// NS shared-memory stages: the consumers hold one or two of them (the stage
// being read and the previous one, whose node data the finished node plane
// needs), the rest is the producer's lead.  RPC = 1: 4 or 5 stages (57 / 72 KB)
// fit 3 CTAs per SM (the default, 5), 6 or 7 stages (86 / 100 KB) fit 2.
// RPC = 2 (two right-hand sides per CTA sharing the q*kappa and d boxes and
// every stencil coefficient): 4 stages (94 KB), 2 CTAs per SM.
template <int NS, int RPC>
__global__ void __launch_bounds__(kThreads + 32, RPC == 2 ? 2 : (NS >= 6 ? 2 : 3))
stream3d_pair_kernel(const __grid_constant__ Stream3Maps maps, int iu, int ium,
                     float *__restrict__ um, Layout L, StepCoef<float> C, float a, float b,
                     const OutSlot *__restrict__ slot, int flags, int zchunk, int *__restrict__ err,
                     RhsSet R)
{
    constexpr int kSE = stage_elems<RPC>();
    extern __shared__ __align__(128) float ring[];
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + NS * kSE);
    uint64_t *empty = full + NS;
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    // the rhs slots vary fastest over the CTAs, so the rhs of one column tile
    // run side by side and share its q*kappa and d through L2; a CTA takes
    // slots g RPC .. g RPC + RPC - 1 of its group g (the present ones)
    const int ngroups = (R.slots + RPC - 1) / RPC;
    const int grp = (int)(blockIdx.x % (unsigned)ngroups);
    int rr[RPC];
    int nr = 0;
#pragma unroll
    for (int q = 0; q < RPC; ++q) {
        int rq;
        if (grp * RPC + q < R.slots && rhs_of_slot(R, grp * RPC + q, rq)) rr[nr++] = rq;
    }
    if (nr == 0) return;
#pragma unroll
    for (int q = 1; q < RPC; ++q)
        if (q >= nr) rr[q] = rr[0];          // an absent second rhs repeats the first (not stored)
    if (smem_u32(ring) & 127u) {              // TMA destinations must be 128-byte aligned
        if (tid == 0) atomicExch(err, 1);
        return;
    }
    const int64_t x0 = (int64_t)(blockIdx.x / (unsigned)ngroups) * kTX;
    const int64_t y0 = (int64_t)blockIdx.y * kTY;
    const int64_t zb = (int64_t)blockIdx.z * zchunk;
    const int64_t ze = min((int64_t)L.nz, zb + zchunk);
    if (zb >= ze) return;
    const int64_t c0 = L.xl + x0 - 1;
    const int xs = (int)(c0 & ~(int64_t)3);
    const int xn = (int)(L.xl + x0);
    const int nplanes = (int)(ze - zb) + 2;

    if (tid == 0) {
        for (int st = 0; st < NS; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[st])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[st])),
                         "r"(kThreads / 32));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    grid_dep_launch();       // the next step may be scheduled as this grid's CTAs retire

    // ---- producer warp ----------------------------------------------------
    if (tid >= kThreads) {
        if (tid == kThreads) {
            // the first NS stages: coefficients before the wait for the previous
            // step, states after it
            const int npre = min(NS, nplanes);
            auto kind_of = [&](int p) { return p == 0 ? 1 : (p == nplanes - 1 ? 2 : 0); };
            for (int p = 0; p < npre; ++p)
                load_stage_coef<RPC>(maps, ring + p * kSE, &full[p], xs, xn, (int)y0,
                                     (int)(zb + p), rr, nr, kind_of(p));
            grid_dep_wait();
            for (int p = 0; p < npre; ++p)
                load_stage_state<RPC>(maps, iu, ium, ring + p * kSE, &full[p], xs, xn, (int)y0,
                                      (int)(zb + p), rr, nr, kind_of(p));
            for (int p = NS; p < nplanes; ++p) {
                const int st = p % NS;
                if (!wait_bounded(&empty[st], (unsigned)(((p / NS) - 1) & 1), &abort_flag)) break;
                float *stage = ring + st * kSE;
                load_stage_coef<RPC>(maps, stage, &full[st], xs, xn, (int)y0, (int)(zb + p), rr,
                                     nr, kind_of(p));
                load_stage_state<RPC>(maps, iu, ium, stage, &full[st], xs, xn, (int)y0,
                                      (int)(zb + p), rr, nr, kind_of(p));
            }
            if (abort_flag) {
                atomicExch(err, 1);
                for (int st = 0; st < NS && st < nplanes; ++st) {
                    const int last = (nplanes - 1 - st) / NS;
                    const unsigned long long t0 = global_ns();
                    while (!mbar_try_wait(&full[st], (unsigned)(last & 1)) &&
                           global_ns() - t0 < kWaitLimitNs) {
                    }
                }
            }
        }
        return;
    }

    // ---- consumer warps: nodes (x, x+1), x = x0 + 2 tx, row y = y0 + ty ----
    grid_dep_wait();         // before any write of a plane the previous step reads
    const int tx = tid & 31, ty = tid >> 5;
    const int lane = tid & 31;
    const int64_t gx = x0 + 2 * tx, gy = y0 + ty;
    const bool rowok = gy < L.ny;
    const bool actA = rowok && gx < L.nx, actB = rowok && gx + 1 < L.nx;
    const float2 cc0 = bc(C.c0), m0 = bc(C.mt[0]);
    const float2 mf[4] = {bc(C.mt[0]), bc(C.mt[1]), bc(C.mt[2]), bc(C.mt[3])};
    const float2 ncf[4] = {bc(0.f), bc(-C.cs[1]), bc(-C.cs[2]), bc(-C.cs[3])};
    const float2 a2 = bc(a), nb2 = bc(-b), ntwo = bc(-2.f);
    int wst = 0;
    unsigned wph = 0;
    // the outcome is made warp-uniform, so that a warp never splits between
    // giving up and going on to the warp-wide release
    auto full_wait_next = [&]() -> bool {
        const bool r = __all_sync(0xffffffffu, wait_bounded(&full[wst], wph, &abort_flag));
        if (++wst == NS) { wst = 0; wph ^= 1u; }
        return r;
    };
    int rst = 0;
    auto release_next = [&]() {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[rst]);
        if (++rst == NS) rst = 0;
    };
    // box offsets: row ty (= node row - 1), column of node x - 1 in the halo boxes,
    // (ty, 2 tx) in the node boxes
    const int uo = ty * kHaloW + 2 * tx + 3;
    const int no = ty * kTX + 2 * tx;
    float *ump[RPC];                                   // u_{j+1} at node zb, per rhs
#pragma unroll
    for (int q = 0; q < RPC; ++q)
        ump[q] = um + rr[q] * R.stride + (zb + 1) * L.plane + (gy + 1) * L.pitch + L.xl + gx;
    int64_t cidx = (zb * L.ny + gy) * L.nx + gx;
    const int64_t cstride = L.ny * L.nx;

    // u_j of one stored plane at row oy as the three pairs (u(x-1+ox), u(x+ox))
    auto load_u = [&](float2 (&w)[3], const float *ubox, int oy) {
        const float *r = ubox + uo + oy * kHaloW;
        const float um1 = r[0];
        const float2 mid = *reinterpret_cast<const float2 *>(r + 1);
        const float up2 = r[3];
        w[0] = f2(um1, mid.x);
        w[1] = mid;
        w[2] = f2(mid.y, up2);
    };
    // sums of q*kappa of one cell plane over the cells shared with the neighbour at
    // (oy, ox) - 1 (-1 keeps the lower cell, +1 the upper, 0 both), same order of
    // additions as the one-node kernel: along x first, then across y
    auto load_k = [&](float2 (&kk)[3][3], const float *stage) {
        const float *r = stage + RPC * kHaloStride + uo;
        float2 kx[2][3];
#pragma unroll
        for (int ay = 0; ay < 2; ++ay) {
            const float km = r[ay * kHaloW];
            const float2 k2 = *reinterpret_cast<const float2 *>(r + ay * kHaloW + 1);
            kx[ay][0] = f2(km, k2.x);
            kx[ay][2] = k2;
            kx[ay][1] = add2(kx[ay][0], kx[ay][2]);
        }
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) {
            kk[0][ox] = kx[0][ox];
            kk[1][ox] = add2(kx[0][ox], kx[1][ox]);
            kk[2][ox] = kx[1][ox];
        }
    };
    // Each stored plane P is read from the ring once: its u_j rows are pushed
    // into the stencil sums of the three node planes it touches -- P + 1 (as
    // its lower plane, with the cell sums of c(P)), P (middle plane, c(P-1) +
    // c(P)) and P - 1 (upper plane, c(P-1)) -- where c(P) is the cell plane
    // stored with P.  A node plane receives its lower, middle and upper terms in
    // that order, each in (oy, ox) order, so the sums are those of the one-node
    // kernel bit for bit.  accL, accM, accU: node planes P + 1, P, P - 1, one
    // set per rhs; every coefficient is computed once and used for each rhs.
    float2 kprev[3][3], kcur[3][3];
#pragma unroll
    for (int oy = 0; oy < 3; ++oy)
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) kprev[oy][ox] = bc(0.f);
    float2 accL[RPC], accM[RPC], accU[RPC];
#pragma unroll
    for (int q = 0; q < RPC; ++q) accL[q] = accM[q] = accU[q] = bc(0.f);
    auto coef = [&](int oz, int oy, int ox, float2 ks) -> float2 {
        const int sh = (oz != 1) + (oy != 1) + (ox != 1);
        return (sh == 0) ? fma2(m0, ks, cc0) : fma2(mf[sh], ks, ncf[sh]);
    };
    // the terms of stored plane `st` for the node planes flagged
    auto push = [&](const float *st, auto doL, auto doM, auto doU) {
        constexpr bool kL = decltype(doL)::value, kM = decltype(doM)::value,
                       kU = decltype(doU)::value;
#pragma unroll
        for (int oy = 0; oy < 3; ++oy) {
            float2 uv[RPC][3];
#pragma unroll
            for (int q = 0; q < RPC; ++q) load_u(uv[q], st + q * kHaloStride, oy);
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) {
                if (kL) {
                    const float2 cL = coef(0, oy, ox, kcur[oy][ox]);
#pragma unroll
                    for (int q = 0; q < RPC; ++q) accL[q] = fma2(cL, uv[q][ox], accL[q]);
                }
                if (kM) {
                    const float2 cM = coef(1, oy, ox, add2(kprev[oy][ox], kcur[oy][ox]));
#pragma unroll
                    for (int q = 0; q < RPC; ++q) accM[q] = fma2(cM, uv[q][ox], accM[q]);
                }
                if (kU) {
                    const float2 cU = coef(2, oy, ox, kprev[oy][ox]);
#pragma unroll
                    for (int q = 0; q < RPC; ++q) accU[q] = fma2(cU, uv[q][ox], accU[q]);
                }
            }
        }
    };
    // node plane of stored plane `sn` complete: update, store, outputs
    auto finish = [&](const float *sn) {
        const float *nd = sn + (RPC + 1) * kHaloStride + no;
        const float2 d = *reinterpret_cast<const float2 *>(nd);
#pragma unroll
        for (int q = 0; q < RPC; ++q) {
            const float *nq = nd + kNodeElems + q * 3 * kNodeElems;
            const float2 fr = *reinterpret_cast<const float2 *>(nq);
            const float2 fi = *reinterpret_cast<const float2 *>(nq + kNodeElems);
            const float2 uprev = *reinterpret_cast<const float2 *>(nq + 2 * kNodeElems);
            const float2 g = fma2(a2, fr, mul2(nb2, fi));
            const float2 t = fma2(ntwo, uprev, add2(accU[q], g));
            const float2 unew = fma2(d, t, uprev);
            if (q < nr) {
                if (actB) {
                    *reinterpret_cast<float2 *>(ump[q]) = unew;
                } else if (actA) {
                    *ump[q] = unew.x;
                }
                if (flags && actA) {
                    const OutSlot *sl = slot + rr[q];
                    if ((flags & 1) && sl->snap_part) {
                        sl->snap_part[2 * cidx] = (double)unew.x;
                        if (actB) sl->snap_part[2 * cidx + 2] = (double)unew.y;
                    }
                    if ((flags & 2) && sl->final_part) {
                        sl->final_part[2 * cidx] = (double)unew.x;
                        if (actB) sl->final_part[2 * cidx + 2] = (double)unew.y;
                    }
                }
            }
            ump[q] += L.plane;
        }
        cidx += cstride;
    };

    // stored planes zb + p, p = 0 .. nplanes - 1; node planes are stored planes
    // 1 .. nplanes - 2.  Plane p feeds node p + 1 if p <= nplanes - 3, node p if
    // 1 <= p <= nplanes - 2, node p - 1 if p >= 2 (which it completes); after
    // plane p the stage of plane p - 1 is no longer needed.
    using T_ = std::true_type;
    using F_ = std::false_type;
    bool ok = true;
    for (int p = 0; p < nplanes; ++p) {
        if (!(ok = full_wait_next())) break;
        const float *st = ring + (p % NS) * kSE;
        if (p < nplanes - 1) load_k(kcur, st);
        const bool hL = p <= nplanes - 3, hM = p >= 1 && p <= nplanes - 2, hU = p >= 2;
        if (hL && hM && hU) push(st, T_{}, T_{}, T_{});
        else if (hL && hM) push(st, T_{}, T_{}, F_{});
        else if (hL && hU) push(st, T_{}, F_{}, T_{});
        else if (hM && hU) push(st, F_{}, T_{}, T_{});
        else if (hL) push(st, T_{}, F_{}, F_{});
        else if (hM) push(st, F_{}, T_{}, F_{});
        else push(st, F_{}, F_{}, T_{});
        if (hU) finish(ring + ((p - 1) % NS) * kSE);
        if (p >= 1) release_next();
#pragma unroll
        for (int q = 0; q < RPC; ++q) {
            accU[q] = accM[q];
            accM[q] = accL[q];
            accL[q] = bc(0.f);
        }
#pragma unroll
        for (int oy = 0; oy < 3; ++oy)
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) kprev[oy][ox] = kcur[oy][ox];
    }
}

}  // namespace

size_t stream3d_pair_smem_bytes(int stages, int rpc)
{
    const int se = (rpc == 2) ? stage_elems<2>() : stage_elems<1>();
    return (size_t)stages * se * sizeof(float) + 2 * stages * sizeof(uint64_t);
}

bool make_stream3d_pair_maps(const Layout &L, float *const planes[6], Stream3Maps *maps, int nrhs)
{
    typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    // node pairs need even columns: the padded layout's x lead must be even
    if (L.d != 3 || (L.xl % 4) != 0 || nrhs < 1) return false;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        (void)cudaGetLastError();
        return false;
    }
    EncodeFn encode = reinterpret_cast<EncodeFn>(fn);
    const cuuint64_t dims[4] = {(cuuint64_t)L.pitch, (cuuint64_t)(L.ny + 2), (cuuint64_t)(L.nz + 2),
                                (cuuint64_t)nrhs};
    const cuuint64_t strides[3] = {(cuuint64_t)(L.pitch * sizeof(float)),
                                   (cuuint64_t)(L.plane * sizeof(float)),
                                   (cuuint64_t)(L.total * sizeof(float))};
    const cuuint32_t halo[4] = {(cuuint32_t)kHaloW, (cuuint32_t)kHaloH, 1, 1};
    const cuuint32_t node[4] = {(cuuint32_t)kTX, (cuuint32_t)kTY, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    float *src[8] = {planes[0], planes[1], planes[2], planes[3], planes[4], planes[5], planes[0],
                     planes[1]};
    for (int i = 0; i < 8; ++i) {
        const cuuint32_t *box = (i < 3) ? halo : node;
        const cuuint32_t rank = (i == 2 || i == 3) ? 3 : 4;     // q*kappa and d are shared
        if (encode(&maps->m[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, (void *)src[i], dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return false;
    }
    const int smem_attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    return cudaFuncSetAttribute(stream3d_pair_kernel<7, 1>, (cudaFuncAttribute)smem_attr,
                                (int)stream3d_pair_smem_bytes(7, 1)) == cudaSuccess &&
           cudaFuncSetAttribute(stream3d_pair_kernel<6, 1>, (cudaFuncAttribute)smem_attr,
                                (int)stream3d_pair_smem_bytes(6, 1)) == cudaSuccess &&
           cudaFuncSetAttribute(stream3d_pair_kernel<5, 1>, (cudaFuncAttribute)smem_attr,
                                (int)stream3d_pair_smem_bytes(5, 1)) == cudaSuccess &&
           cudaFuncSetAttribute(stream3d_pair_kernel<4, 1>, (cudaFuncAttribute)smem_attr,
                                (int)stream3d_pair_smem_bytes(4, 1)) == cudaSuccess &&
           cudaFuncSetAttribute(stream3d_pair_kernel<4, 2>, (cudaFuncAttribute)smem_attr,
                                (int)stream3d_pair_smem_bytes(4, 2)) == cudaSuccess;
}

int stream3d_pair_zchunk(const Layout &L, int stages, int rpc)
{
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = ((L.nx + kTX - 1) / kTX) * ((L.ny + kTY - 1) / kTY);
    int64_t zc = 64;
    const int per_sm = (rpc == 2 || stages >= 6) ? 2 : 3;
    while (zc > 16 && tiles * ((L.nz + zc - 1) / zc) < per_sm * nsm) zc /= 2;
    if (zc > L.nz) zc = L.nz;
    return (int)zc;
}

void launch_stream3d_pair(const Stream3Maps &maps, int from, const Layout &L, float *um,
                          const StepCoef<float> &C, float a, float b, const OutSlot *slot,
                          int flags, int zchunk, int stages, int *err, cudaStream_t s,
                          const RhsSet &R, bool overlap, int rpc)
{
    const int iu = from ? 1 : 0, ium = from ? 6 : 7;
    const int groups = (rpc == 2) ? (R.slots + 1) / 2 : R.slots;
    dim3 grd((unsigned)(((L.nx + kTX - 1) / kTX) * groups), (unsigned)((L.ny + kTY - 1) / kTY),
             (unsigned)((L.nz + zchunk - 1) / zchunk));
    if (rpc == 2)
        launch_ex(stream3d_pair_kernel<4, 2>, grd, kThreads + 32, stream3d_pair_smem_bytes(4, 2),
                  s, overlap, maps, iu, ium, um, L, C, a, b, slot, flags, zchunk, err, R);
    else if (stages == 7)
        launch_ex(stream3d_pair_kernel<7, 1>, grd, kThreads + 32, stream3d_pair_smem_bytes(7, 1),
                  s, overlap, maps, iu, ium, um, L, C, a, b, slot, flags, zchunk, err, R);
    else if (stages == 5)
        launch_ex(stream3d_pair_kernel<5, 1>, grd, kThreads + 32, stream3d_pair_smem_bytes(5, 1),
                  s, overlap, maps, iu, ium, um, L, C, a, b, slot, flags, zchunk, err, R);
    else if (stages == 4)
        launch_ex(stream3d_pair_kernel<4, 1>, grd, kThreads + 32, stream3d_pair_smem_bytes(4, 1),
                  s, overlap, maps, iu, ium, um, L, C, a, b, slot, flags, zchunk, err, R);
    else
        launch_ex(stream3d_pair_kernel<6, 1>, grd, kThreads + 32, stream3d_pair_smem_bytes(6, 1),
                  s, overlap, maps, iu, ium, um, L, C, a, b, slot, flags, zchunk, err, R);
    ++g_launches;
}

}  // namespace htd
