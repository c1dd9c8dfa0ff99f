// 3-D recurrence step streamed through shared memory by TMA (FP32).
//
// One step of I_acd (Def. of I_acd) with Table 1's windowed forcing, as in
// step3d_kernel, but organised for HBM streaming: each CTA owns a 32 x 8 tile of
// (x, y) columns and a chunk of z planes.  A producer warp keeps a ring of
// kStages shared-memory stages filled with cp.async.bulk.tensor.3d copies
// ("full" mbarrier per stage); the 8 consumer warps release a stage with one
// arrival each on its "empty" mbarrier, so no CTA-wide barrier is needed per
// plane.  A stage holds, for
// one stored plane p, the u_j box and the q*kappa box (34 x 10 nodes/cells with
// the x-y halo, starting at a 16-byte aligned column) and the exact 32 x 8 boxes
// of d, Re F, Im F and u_{j-1}.  Node plane iz reads stored planes iz, iz+1,
// iz+2 of u_j (kept in rotating register windows), cells of stored planes iz and
// iz+1, and the node data of stored plane iz+1; u_{j+1} is stored straight to
// global memory over u_{j-1}.  Every wait is time-bounded; a CTA that gives up
// raises an abort flag that ends all its warps' waits and sets the error word.
// The per-node arithmetic is that of step3d_kernel (same expression, order).
#include <cuda.h>
#include <cuda_runtime.h>

#include "htd_internal.h"

namespace htd {

namespace {

constexpr int kStages = 6;
constexpr int kThreads = 256;                               // consumer threads: one per column
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

// Tile geometry: TXW x TYH columns (TXW * TYH = 256).  The u / kappa box is
// TXW + 2 (+ up to 3 for the 16-byte alignment) wide, rounded to 8 floats, and
// TYH + 2 high; node boxes are exactly TXW x TYH.
template <int TXW, int TYH>
struct Geo {
    static_assert(TXW * TYH == kThreads, "one consumer thread per column");
    static constexpr int kTX = TXW, kTY = TYH;
    static constexpr int kHaloW = ((TXW + 5 + 7) / 8) * 8;
    static constexpr int kHaloH = TYH + 2;
    static constexpr int kHaloElems = kHaloW * kHaloH;
    static constexpr int kHaloStride = ((kHaloElems * 4 + 127) / 128) * 32;   // 128-byte padded
    static constexpr int kNodeElems = TXW * TYH;
    static constexpr int kStageElems = 2 * kHaloStride + 4 * kNodeElems;
    static constexpr unsigned kStageTxBytes = (2 * kHaloElems + 4 * kNodeElems) * 4;
};

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

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// issue the six copies of stored plane p into stage `st`
template <class G>
__device__ __forceinline__ void load_stage(const Stream3Maps &maps, int iu, int ium, float *stage,
                                           uint64_t *bar, int xs, int xn, int y0, int p)
{
    constexpr int kHaloStride = G::kHaloStride, kNodeElems = G::kNodeElems;
    constexpr unsigned kStageTxBytes = G::kStageTxBytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(kStageTxBytes)
                 : "memory");
    tma_load_3d(stage, &maps.m[iu], xs, y0, p, bar);                                // u_j, halo
    tma_load_3d(stage + kHaloStride, &maps.m[2], xs, y0, p, bar);                    // kappa, halo
    tma_load_3d(stage + 2 * kHaloStride, &maps.m[3], xn, y0 + 1, p, bar);            // d
    tma_load_3d(stage + 2 * kHaloStride + kNodeElems, &maps.m[4], xn, y0 + 1, p, bar);      // Re F
    tma_load_3d(stage + 2 * kHaloStride + 2 * kNodeElems, &maps.m[5], xn, y0 + 1, p, bar);  // Im F
    tma_load_3d(stage + 2 * kHaloStride + 3 * kNodeElems, &maps.m[ium], xn, y0 + 1, p, bar); // u_{j-1}
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bounded wait for the completion of the phase with parity `phase`; gives up
// (and raises the CTA's abort flag) after kWaitLimitNs, or at once if another
// warp already gave up
__device__ __forceinline__ bool wait_bounded(uint64_t *bar, unsigned phase, volatile int *abort_flag)
{
    if (mbar_try_wait(bar, phase)) return true;           // fast path: no timer read
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

template <int TXW, int TYH>
__global__ void __launch_bounds__(kThreads + 32, 2)
stream3d_kernel(const __grid_constant__ Stream3Maps maps, int iu, int ium, float *__restrict__ um,
                Layout L, StepCoef<float> C, float a, float b, const OutSlot *__restrict__ slot,
                int flags, int zchunk, int *__restrict__ err)
{
    using G = Geo<TXW, TYH>;
    constexpr int kTX = G::kTX, kTY = G::kTY, kHaloW = G::kHaloW, kHaloStride = G::kHaloStride;
    constexpr int kNodeElems = G::kNodeElems, kStageElems = G::kStageElems;
    // dynamic shared memory: the ring of stages (128-byte aligned boxes), then
    // the full and empty mbarriers
    extern __shared__ __align__(128) float ring[];
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + kStages * kStageElems);
    uint64_t *empty = full + kStages;
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    // TMA destinations must be 128-byte aligned; refuse to run otherwise
    if (smem_u32(ring) & 127u) {
        if (tid == 0) atomicExch(err, 1);
        return;
    }
    const int64_t x0 = (int64_t)blockIdx.x * kTX, y0 = (int64_t)blockIdx.y * kTY;
    const int64_t zb = (int64_t)blockIdx.z * zchunk;
    const int64_t ze = min((int64_t)L.nz, zb + zchunk);
    if (zb >= ze) return;
    // u / kappa box: stored column of (x0 - 1) rounded down to 16 bytes
    const int64_t c0 = L.xl + x0 - 1;
    const int xs = (int)(c0 & ~(int64_t)3);
    const int off = (int)(c0 - xs);
    const int xn = (int)(L.xl + x0);                 // node boxes start 128-byte aligned
    const int nplanes = (int)(ze - zb) + 2;          // stored planes zb .. ze+1
    const int nq = nplanes - 2;                      // node planes zb .. ze-1

    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[st])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[st])),
                         "r"(kThreads / 32));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();

    // ---- producer warp: one lane streams the planes through the ring --------
    if (tid >= kThreads) {
        if (tid == kThreads) {
            for (int p = 0; p < nplanes; ++p) {
                const int st = p % kStages;
                // the stage's previous plane (p - kStages) must have been released
                if (p >= kStages && !wait_bounded(&empty[st], (unsigned)(((p / kStages) - 1) & 1),
                                                  &abort_flag))
                    break;
                load_stage<G>(maps, iu, ium, ring + st * kStageElems, &full[st], xs, xn, (int)y0,
                              (int)(zb + p));
            }
            if (abort_flag) {
                atomicExch(err, 1);
                // wait (bounded) for the copies still in flight before leaving
                for (int st = 0; st < kStages && st < nplanes; ++st) {
                    const int last = ((nplanes - 1 - st) / kStages);   // last use of this stage
                    const unsigned long long t0 = global_ns();
                    while (!mbar_try_wait(&full[st], (unsigned)(last & 1)) &&
                           global_ns() - t0 < kWaitLimitNs) {
                    }
                }
            }
        }
        return;
    }

    // ---- consumer warps ---------------------------------------------------
    const int tx = tid & (kTX - 1), ty = tid / kTX;
    const int lane = tid & 31;
    const int64_t gx = x0 + tx, gy = y0 + ty;
    const bool active = gx < L.nx && gy < L.ny;
    // coefficients in registers: c0, cs_s (s = 1..3), M_s (s = 0..3)
    const float cc0 = C.c0, cs1 = C.cs[1], cs2 = C.cs[2], cs3 = C.cs[3];
    const float m0 = C.mt[0], m1 = C.mt[1], m2 = C.mt[2], m3 = C.mt[3];
    // next plane to wait for: its stage and the parity of its use of that stage
    int wst = 0;
    unsigned wph = 0;
    auto full_wait_next = [&]() -> bool {
        const bool r = wait_bounded(&full[wst], wph, &abort_flag);
        if (++wst == kStages) { wst = 0; wph ^= 1u; }
        return r;
    };
    int rst = 0;                                                // next stage to release
    auto release_next = [&]() {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[rst]);
        if (++rst == kStages) rst = 0;
    };

    // register windows: u_j of three stored planes (9 values each) and, per cell
    // plane, the sums of q*kappa over the cells shared with the neighbour at
    // (oy, ox) - 1 within that plane (-1 keeps the lower cell, +1 the upper, 0 both)
    float wa[3][3], wb[3][3], wc[3][3];
    float ka[3][3], kb[3][3], kc[3][3];
    const int uo = ty * kHaloW + tx + off;                     // box offset of (ty-1, tx-1)
    float *ump = um + (zb + 1) * L.plane + (gy + 1) * L.pitch + L.xl + gx;   // u_{j+1} at node zb
    int64_t cidx = (zb * L.ny + gy) * L.nx + gx;               // compact index at node zb
    const int64_t cstride = L.ny * L.nx;
    auto load_u = [&](float (&w)[3][3], int st) {
        const int b0 = st * kStageElems + uo;
#pragma unroll
        for (int oy = 0; oy < 3; ++oy)
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) w[oy][ox] = ring[b0 + oy * kHaloW + ox];
    };
    auto load_k = [&](float (&kk)[3][3], int st) {
        const int b0 = st * kStageElems + kHaloStride + uo;
        const float k00 = ring[b0], k01 = ring[b0 + 1], k10 = ring[b0 + kHaloW],
                    k11 = ring[b0 + kHaloW + 1];
        const float r0 = k00 + k01, r1 = k10 + k11;
        kk[0][0] = k00; kk[0][1] = r0; kk[0][2] = k01;
        kk[1][0] = k00 + k10; kk[1][1] = r0 + r1; kk[1][2] = k01 + k11;
        kk[2][0] = k10; kk[2][1] = r1; kk[2][2] = k11;
    };
    // one node: planes (lo, mid, hi) = stored iz, iz+1, iz+2; cells (kl, kh) = stored iz,
    // iz+1; node data from stage st1 (stored iz+1)
    auto update = [&](const float (&lo)[3][3], const float (&mid)[3][3], const float (&hi)[3][3],
                      const float (&kl)[3][3], const float (&kh)[3][3], int st1) {
        const float cf[4] = {0.f, cs1, cs2, cs3};
        const float mf[4] = {m0, m1, m2, m3};
        float acc = 0.f;
#pragma unroll
        for (int oz = 0; oz < 3; ++oz)
#pragma unroll
            for (int oy = 0; oy < 3; ++oy)
#pragma unroll
                for (int ox = 0; ox < 3; ++ox) {
                    const int sh = (oz != 1) + (oy != 1) + (ox != 1);
                    const float ks = (oz == 0) ? kl[oy][ox] : (oz == 2) ? kh[oy][ox]
                                                                      : kl[oy][ox] + kh[oy][ox];
                    const float uv = (oz == 0) ? lo[oy][ox] : (oz == 1) ? mid[oy][ox] : hi[oy][ox];
                    const float coef = (sh == 0) ? cc0 + m0 * ks : mf[sh] * ks - cf[sh];
                    acc += coef * uv;
                }
        const int nb = st1 * kStageElems + 2 * kHaloStride + tid;
        const float d = ring[nb], fr = ring[nb + kNodeElems], fi = ring[nb + 2 * kNodeElems];
        const float uprev = ring[nb + 3 * kNodeElems];
        if (active) {
            const float g = a * fr - b * fi;
            const float unew = d * (acc + g - 2.f * uprev) + uprev;
            *ump = unew;
            if (flags) {
                if ((flags & 1) && slot->snap_part) slot->snap_part[2 * cidx] = (double)unew;
                if ((flags & 2) && slot->final_part) slot->final_part[2 * cidx] = (double)unew;
            }
        }
        ump += L.plane;
        cidx += cstride;
    };

    bool ok = full_wait_next() && full_wait_next();             // stored planes zb, zb + 1
    if (ok) {
        load_u(wa, 0);
        load_u(wb, 1);
        load_k(ka, 0);
        release_next();                                        // plane zb's node data is unused
    }
    int st1 = 1, st2 = 2;                                      // stages of stored iz+1, iz+2
    // node plane iz reads u of stored iz+2 and cells and node data of stored iz+1;
    // afterwards stored plane iz+1 is no longer needed
    auto plane = [&](float (&lo)[3][3], float (&mid)[3][3], float (&hi)[3][3],
                     float (&kl)[3][3], float (&kh)[3][3]) -> bool {
        if (!full_wait_next()) return false;
        load_u(hi, st2);
        load_k(kh, st1);
        update(lo, mid, hi, kl, kh, st1);
        release_next();
        st1 = st2;
        if (++st2 == kStages) st2 = 0;
        return true;
    };
    for (int q = 0; ok && q < nq; q += 3) {
        // windows rotate with period 3: u planes (wa, wb, wc), cell planes (ka, kb, kc)
        if (!(ok = plane(wa, wb, wc, ka, kb))) break;
        if (q + 1 >= nq) break;
        if (!(ok = plane(wb, wc, wa, kb, kc))) break;
        if (q + 2 >= nq) break;
        if (!(ok = plane(wc, wa, wb, kc, ka))) break;
    }
    // the last stored plane (ze+1) is only read for u; release it for symmetry
    if (ok) release_next();

}


template <int TXW, int TYH>
size_t smem_bytes_t()
{
    return (size_t)kStages * Geo<TXW, TYH>::kStageElems * sizeof(float) +
           2 * kStages * sizeof(uint64_t);
}

template <int TXW, int TYH>
bool make_maps_t(const Layout &L, float *const planes[6], Stream3Maps *maps)
{
    using G = Geo<TXW, TYH>;
    typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    if (L.d != 3 || (L.xl % 4) != 0) return false;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        (void)cudaGetLastError();
        return false;
    }
    EncodeFn encode = reinterpret_cast<EncodeFn>(fn);
    const cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)(L.ny + 2), (cuuint64_t)(L.nz + 2)};
    const cuuint64_t strides[2] = {(cuuint64_t)(L.pitch * sizeof(float)),
                                   (cuuint64_t)(L.plane * sizeof(float))};
    const cuuint32_t halo[3] = {(cuuint32_t)G::kHaloW, (cuuint32_t)G::kHaloH, 1};
    const cuuint32_t node[3] = {(cuuint32_t)G::kTX, (cuuint32_t)G::kTY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    // planes: u0, u1, kappa, d, Re F, Im F
    float *src[8] = {planes[0], planes[1], planes[2], planes[3], planes[4], planes[5], planes[0],
                     planes[1]};
    for (int i = 0; i < 8; ++i) {
        const cuuint32_t *box = (i < 3) ? halo : node;
        if (encode(&maps->m[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)src[i], dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return false;
    }
    return cudaFuncSetAttribute(stream3d_kernel<TXW, TYH>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes_t<TXW, TYH>()) == cudaSuccess;
}

template <int TXW, int TYH>
int zchunk_t(const Layout &L)
{
    int dev = 0, nsm = 1, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, stream3d_kernel<TXW, TYH>, kThreads + 32,
                                                      smem_bytes_t<TXW, TYH>()) != cudaSuccess ||
        occ < 1) {
        (void)cudaGetLastError();
        occ = 1;
    }
    // 64-plane chunks (measured on 256^3: 64 best; 16 about 8% and 256 about 30%
    // slower); smaller grids are split so that every SM still gets work
    (void)occ;
    const int64_t tiles = ((L.nx + TXW - 1) / TXW) * ((L.ny + TYH - 1) / TYH);
    int64_t zc = 64;
    while (zc > 16 && tiles * ((L.nz + zc - 1) / zc) < nsm) zc /= 2;
    if (zc > L.nz) zc = L.nz;
    return (int)zc;
}

template <int TXW, int TYH>
void launch_t(const Stream3Maps &maps, int iu, int ium, const Layout &L, float *um,
              const StepCoef<float> &C, float a, float b, const OutSlot *slot, int flags,
              int zchunk, int *err, cudaStream_t s)
{
    dim3 grd((unsigned)((L.nx + TXW - 1) / TXW), (unsigned)((L.ny + TYH - 1) / TYH),
             (unsigned)((L.nz + zchunk - 1) / zchunk));
    stream3d_kernel<TXW, TYH><<<grd, kThreads + 32, smem_bytes_t<TXW, TYH>(), s>>>(
        maps, iu, ium, um, L, C, a, b, slot, flags, zchunk, err);
}

}  // namespace

// tile shapes: 0 = 32 x 8, 1 = 64 x 4, 2 = 128 x 2
bool make_stream3d_maps(const Layout &L, int shape, float *const planes[6], Stream3Maps *maps)
{
    switch (shape) {
    case 1: return make_maps_t<64, 4>(L, planes, maps);
    case 2: return make_maps_t<128, 2>(L, planes, maps);
    default: return make_maps_t<32, 8>(L, planes, maps);
    }
}

int stream3d_zchunk(const Layout &L, int shape)
{
    switch (shape) {
    case 1: return zchunk_t<64, 4>(L);
    case 2: return zchunk_t<128, 2>(L);
    default: return zchunk_t<32, 8>(L);
    }
}

void launch_stream3d(const Stream3Maps &maps, int from, int shape, const Layout &L, float *um,
                     const StepCoef<float> &C, float a, float b, const OutSlot *slot, int flags,
                     int zchunk, int *err, cudaStream_t s)
{
    // from = 0: u_j in u0, u_{j-1} (overwritten) in u1; from = 1: the other way round
    const int iu = from ? 1 : 0, ium = from ? 6 : 7;
    switch (shape) {
    case 1: launch_t<64, 4>(maps, iu, ium, L, um, C, a, b, slot, flags, zchunk, err, s); break;
    case 2: launch_t<128, 2>(maps, iu, ium, L, um, C, a, b, slot, flags, zchunk, err, s); break;
    default: launch_t<32, 8>(maps, iu, ium, L, um, C, a, b, slot, flags, zchunk, err, s); break;
    }
    ++g_launches;
}

}  // namespace htd
