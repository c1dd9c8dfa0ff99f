// 3-D recurrence step streamed through shared memory by TMA (FP32).
//
// One step of I_acd (Def. of I_acd) with Table 1's windowed forcing, as in
// step3d_kernel, but organised for HBM streaming: each CTA owns a 32 x 8 tile of
// (x, y) columns and a chunk of z planes.  Thread 0 keeps a ring of kStages
// shared-memory stages filled kStages - 3 planes ahead with
// cp.async.bulk.tensor.3d copies (one mbarrier per stage); a stage holds, for
// one stored plane p, the u_j box and the q*kappa box (34 x 10 nodes/cells with
// the x-y halo, starting at a 16-byte aligned column) and the exact 32 x 8 boxes
// of d, Re F, Im F and u_{j-1}.  Node plane iz reads stored planes iz, iz+1,
// iz+2 of u_j (kept as a 3x3x3 register window), cells of stored planes iz and
// iz+1, and the node data of stored plane iz+1; u_{j+1} is stored straight to
// global memory over u_{j-1}.  After a plane, __syncthreads frees the oldest
// stage and thread 0 refills it.  The per-node arithmetic is that of
// step3d_kernel (same expression, same order).
#include <cuda.h>
#include <cuda_runtime.h>

#include "htd_internal.h"

namespace htd {

namespace {

constexpr int kTX = 32, kTY = 8, kThreads = kTX * kTY;
constexpr int kStages = 6;
constexpr int kHaloW = 40;     // u / kappa box width (34 needed + alignment), FP32
constexpr int kHaloH = kTY + 2;
constexpr int kHaloElems = kHaloW * kHaloH;                 // 400 floats copied
constexpr int kHaloStride = ((kHaloElems * 4 + 127) / 128) * 32;   // padded to 128 bytes
constexpr int kNodeElems = kTX * kTY;                       // 256 floats (1 KB)
constexpr int kStageElems = 2 * kHaloStride + 4 * kNodeElems;
constexpr unsigned kStageTxBytes = (2 * kHaloElems + 4 * kNodeElems) * 4;
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
__device__ __forceinline__ void load_stage(const Stream3Maps &maps, int iu, int ium, float *stage,
                                           uint64_t *bar, int xs, int xn, int y0, int p)
{
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

__global__ void __launch_bounds__(kThreads)
stream3d_kernel(const __grid_constant__ Stream3Maps maps, int iu, int ium, float *__restrict__ um,
                Layout L, StepCoef<float> C, float a, float b, const OutSlot *__restrict__ slot,
                int flags, int zchunk, int *__restrict__ err)
{
    extern __shared__ unsigned char smem_raw[];
    const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127;
    float *ring = reinterpret_cast<float *>(base);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + (size_t)kStages * kStageElems * sizeof(float));

    const int tid = threadIdx.x;
    const int tx = tid & (kTX - 1), ty = tid / kTX;
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

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int q = 0; q < kStages && q < nplanes; ++q)
            load_stage(maps, iu, ium, ring + (size_t)q * kStageElems, &bars[q], xs, xn, (int)y0,
                       (int)(zb + q));
    }
    __syncthreads();

    const int64_t gx = x0 + tx, gy = y0 + ty;
    const bool active = gx < L.nx && gy < L.ny;
    bool ok = true;
    // wait for stored plane zb + q (q-th plane of this chunk), bounded
    auto wait_plane = [&](int q) {
        const unsigned phase = (unsigned)((q / kStages) & 1);
        const unsigned long long t0 = global_ns();
        while (!mbar_try_wait(&bars[q % kStages], phase)) {
            if (global_ns() - t0 > kWaitLimitNs) { ok = false; break; }
        }
    };

    float w[3][3][3];
    float k[2][2][2];
    wait_plane(0);
    wait_plane(1);
    {
        const float *u0s = ring;                                 // stored plane zb
        const float *u1s = ring + kStageElems;                   // stored plane zb + 1
#pragma unroll
        for (int oy = 0; oy < 3; ++oy)
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) {
                w[0][oy][ox] = u0s[(ty + oy) * kHaloW + tx + off + ox];
                w[1][oy][ox] = u1s[(ty + oy) * kHaloW + tx + off + ox];
            }
        const float *k0s = ring + kHaloStride;
#pragma unroll
        for (int ay = 0; ay < 2; ++ay)
#pragma unroll
            for (int ax = 0; ax < 2; ++ax) k[0][ay][ax] = k0s[(ty + ay) * kHaloW + tx + off + ax];
    }

    bool failed = false;                                       // uniform across the CTA
    for (int q = 0; q + 2 < nplanes; ++q) {
        const int64_t iz = zb + q;                             // node plane
        wait_plane(q + 2);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const float *s1 = ring + (size_t)((q + 1) % kStages) * kStageElems;   // stored iz + 1
        const float *s2 = ring + (size_t)((q + 2) % kStages) * kStageElems;   // stored iz + 2
#pragma unroll
        for (int oy = 0; oy < 3; ++oy)
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) w[2][oy][ox] = s2[(ty + oy) * kHaloW + tx + off + ox];
#pragma unroll
        for (int ay = 0; ay < 2; ++ay)
#pragma unroll
            for (int ax = 0; ax < 2; ++ax)
                k[1][ay][ax] = s1[kHaloStride + (ty + ay) * kHaloW + tx + off + ax];
        const float d = s1[2 * kHaloStride + tid];
        const float fr = s1[2 * kHaloStride + kNodeElems + tid];
        const float fi = s1[2 * kHaloStride + 2 * kNodeElems + tid];
        const float uprev = s1[2 * kHaloStride + 3 * kNodeElems + tid];
        // sums of kappa over the cells shared by the node and its neighbour at
        // offset o - 1 (o in 0..2 per axis): -1 keeps the lower cell, +1 the upper, 0 both
        float kx[2][2][3];
#pragma unroll
        for (int az = 0; az < 2; ++az)
#pragma unroll
            for (int ay = 0; ay < 2; ++ay) {
                kx[az][ay][0] = k[az][ay][0];
                kx[az][ay][1] = k[az][ay][0] + k[az][ay][1];
                kx[az][ay][2] = k[az][ay][1];
            }
        float kxy[2][3][3];
#pragma unroll
        for (int az = 0; az < 2; ++az)
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) {
                kxy[az][0][ox] = kx[az][0][ox];
                kxy[az][1][ox] = kx[az][0][ox] + kx[az][1][ox];
                kxy[az][2][ox] = kx[az][1][ox];
            }
        float acc = 0.f;
#pragma unroll
        for (int oz = 0; oz < 3; ++oz)
#pragma unroll
            for (int oy = 0; oy < 3; ++oy)
#pragma unroll
                for (int ox = 0; ox < 3; ++ox) {
                    const int s = (oz != 1) + (oy != 1) + (ox != 1);
                    const float ks = (oz == 0) ? kxy[0][oy][ox]
                                   : (oz == 2) ? kxy[1][oy][ox] : kxy[0][oy][ox] + kxy[1][oy][ox];
                    const float coef = (s == 0) ? C.c0 + C.mt[0] * ks : C.mt[s] * ks - C.cs[s];
                    acc += coef * w[oz][oy][ox];
                }
        if (active) {
            const float g = a * fr - b * fi;
            const float unew = d * (acc + g - 2.f * uprev) + uprev;
            um[(iz + 1) * L.plane + (gy + 1) * L.pitch + L.xl + gx] = unew;
            if (flags) {
                const int64_t c = (iz * L.ny + gy) * L.nx + gx;
                if ((flags & 1) && slot->snap_part) slot->snap_part[2 * c] = (double)unew;
                if ((flags & 2) && slot->final_part) slot->final_part[2 * c] = (double)unew;
            }
        }
#pragma unroll
        for (int oy = 0; oy < 3; ++oy)
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) {
                w[0][oy][ox] = w[1][oy][ox];
                w[1][oy][ox] = w[2][oy][ox];
            }
#pragma unroll
        for (int ay = 0; ay < 2; ++ay)
#pragma unroll
            for (int ax = 0; ax < 2; ++ax) k[0][ay][ax] = k[1][ay][ax];
        // the stage of stored plane iz is no longer read: refill it with plane iz + kStages
        __syncthreads();
        if (tid == 0 && q + kStages < nplanes)
            load_stage(maps, iu, ium, ring + (size_t)(q % kStages) * kStageElems,
                       &bars[q % kStages], xs, xn, (int)y0, (int)(zb + q + kStages));
    }
    if (failed) {
        if (tid == 0) atomicExch(err, 1);
        // wait (bounded) for the copies still in flight before the CTA exits
        if (tid == 0) {
            for (int q = 0; q < nplanes && q < kStages; ++q) {
                const unsigned long long t0 = global_ns();
                while (!mbar_try_wait(&bars[q], 0) && global_ns() - t0 < kWaitLimitNs) {}
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t stream3d_smem_bytes()
{
    return (size_t)kStages * kStageElems * sizeof(float) + kStages * sizeof(uint64_t) + 128;
}

// Tensor maps: [0] u0 halo box, [1] u1 halo box, [2] kappa halo box, [3] d,
// [4] Re F, [5] Im F, [6] u0 node box, [7] u1 node box (3-D: pitch x rows x planes).
bool make_stream3d_maps(const Layout &L, float *const planes[6], Stream3Maps *maps)
{
    typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    if (L.d != 3 || (L.xl % kTX) != 0) return false;
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
    const cuuint32_t halo[3] = {(cuuint32_t)kHaloW, (cuuint32_t)kHaloH, 1};
    const cuuint32_t node[3] = {(cuuint32_t)kTX, (cuuint32_t)kTY, 1};
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
    return cudaFuncSetAttribute(stream3d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stream3d_smem_bytes()) == cudaSuccess;
}

int stream3d_zchunk(const Layout &L)
{
    int dev = 0, nsm = 1, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, stream3d_kernel, kThreads,
                                                      stream3d_smem_bytes()) != cudaSuccess ||
        occ < 1) {
        (void)cudaGetLastError();
        occ = 1;
    }
    const int64_t tiles = ((L.nx + kTX - 1) / kTX) * ((L.ny + kTY - 1) / kTY);
    int64_t chunks = ((int64_t)nsm * occ) / tiles;
    if (chunks < 1) chunks = 1;
    if (chunks > L.nz) chunks = L.nz;
    return (int)((L.nz + chunks - 1) / chunks);
}

void launch_stream3d(const Stream3Maps &maps, int from, const Layout &L, float *um,
                     const StepCoef<float> &C, float a, float b, const OutSlot *slot, int flags,
                     int zchunk, int *err, cudaStream_t s)
{
    // from = 0: u_j in u0, u_{j-1} (overwritten) in u1; from = 1: the other way round
    const int iu = from ? 1 : 0, ium = from ? 6 : 7;
    dim3 grd((unsigned)((L.nx + kTX - 1) / kTX), (unsigned)((L.ny + kTY - 1) / kTY),
             (unsigned)((L.nz + zchunk - 1) / zchunk));
    stream3d_kernel<<<grd, kThreads, stream3d_smem_bytes(), s>>>(maps, iu, ium, um, L, C, a, b, slot,
                                                                 flags, zchunk, err);
    ++g_launches;
}

}  // namespace htd
