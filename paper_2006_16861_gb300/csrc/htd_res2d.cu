// Resident-grid 2-D recurrence (FP32, node pairs): the whole grid stays in
// shared memory, spread over the SMs, for all T n_P steps of a run.
//
// One cooperative launch runs a whole preconditioner run (Def. of I_acd with
// Table 1's windowed forcing and read-out).  The grid is cut into ntx x nty
// tiles of W x H nodes, one CTA per tile and at most one CTA per SM, every CTA
// resident at once.  A CTA loads its tile's q*kappa cells, d and forcing once,
// keeps both recurrence states in shared memory with a one-node ring around
// the tile, and in every step
//  - computes the new state of its edge nodes and publishes each edge value
//    to a global exchange buffer as one 64-bit word (float bits | tag << 32,
//    tag = index of the state + 1; one buffer per state parity);
//  - computes its interior nodes in row strips with a 3 x 3 register window,
//    while the threads that had edge work fetch the neighbours' edges of the
//    new state into the ring, re-reading a word until it carries the expected
//    tag (bounded by the handle's wait limit);
//  - passes one CTA barrier.
// Each exchanged value carries its own tag and moves as one 64-bit access,
// so no fence has to order data before a flag.  A CTA cannot run more than one
// step ahead of a neighbour (it needs the neighbour's edges of the previous
// state), so two buffers per tile suffice; they are zeroed before every run
// (tag 0 is never expected).  Nothing else touches global memory between the
// first load and the two output steps; no CTA waits for another except
// through these words, and a CTA whose wait runs out sets the handle's error
// word, which every other waiting CTA polls, so that all of them return.
//
// Per node the arithmetic is that of step2d_kernel and of the blocked kernels
// (stencil2d, the same expression in the same order), so the results are
// bit-identical to theirs.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "htd_internal.h"

namespace htd {

namespace {

constexpr int kResThreads = 768;

__device__ __forceinline__ float2 pr(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }

__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// one exchanged word: read and written whole, at GPU scope (not cached in L1)
__device__ __forceinline__ unsigned long long ld_word(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_word(unsigned long long *p, float v, unsigned tag)
{
    const unsigned long long w = ((unsigned long long)tag << 32) | __float_as_uint(v);
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__host__ __device__ constexpr size_t res2d_floats(int W, int H)
{
    return 3 * (size_t)(H + 2) * (W + 4) + 3 * (size_t)H * W;
}

// Shared memory (floats): the states U0, U1 and the cells K, each (H + 2) rows
// of SW = W + 4 columns -- node (lx, ly) at row ly + 1, column lx + 2, so that
// the pair (lx, lx + 1), lx even, is 8-byte aligned; cell (cx, cy) (lower
// corner node) at the place of node (cx, cy) -- then d, Re F, Im F of the
// nodes, H x W each.  Exchange buffer of a tile and parity (E = 2W + 2H
// words): bottom row [0, W), top row [W, 2W), left column [2W, 2W + H), right
// column [2W + H, 2W + 2H).
template <int RPT>
__global__ void __launch_bounds__(kResThreads, 1)
res2d_kernel(const float *__restrict__ kap, const float *__restrict__ dco,
             const float *__restrict__ fre, const float *__restrict__ fim, Layout L,
             StepCoef<float> C, const float2 *__restrict__ ab, int nsteps, int jim, int jfin,
             const OutSlot *__restrict__ slot, unsigned long long *__restrict__ xbuf,
             int *__restrict__ err, int W, int H)
{
    extern __shared__ __align__(16) float sm[];
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const int tx = blockIdx.x, ty = blockIdx.y;
    const int ntx = gridDim.x, nty = gridDim.y;
    const int64_t x0 = (int64_t)tx * W, y0 = (int64_t)ty * H;
    const int w = (int)min((int64_t)W, L.nx - x0);
    const int h = (int)min((int64_t)H, L.ny - y0);
    const int SW = W + 4;
    const int NA = (H + 2) * SW;
    float *U0 = sm, *U1 = sm + NA, *K = sm + 2 * NA;
    float *D = sm + 3 * NA, *FR = D + H * W, *FI = FR + H * W;
    const int E = 2 * W + 2 * H;
    unsigned long long *mine = xbuf + (size_t)(ty * ntx + tx) * 2 * E;

    if (tid == 0) s_abort = 0;
    for (int i = tid; i < 2 * NA; i += kResThreads) sm[i] = 0.f;
    for (int i = tid; i < NA; i += kResThreads) {
        const int cy = i / SW - 1, cx = i % SW - 2;
        float v = 0.f;
        if (cx >= -1 && cx < w && cy >= -1 && cy < h)
            v = kap[(y0 + cy + 1) * L.pitch + L.xl + x0 + cx];
        K[i] = v;
    }
    for (int i = tid; i < H * W; i += kResThreads) {
        const int ly = i / W, lx = i % W;
        float dv = 0.f, fr = 0.f, fi = 0.f;
        if (lx < w && ly < h) {
            const int64_t g = (y0 + ly + 1) * L.pitch + L.xl + x0 + lx;
            dv = dco[g];
            fr = fre[g];
            fi = fim[g];
        }
        D[i] = dv;
        FR[i] = fr;
        FI[i] = fi;
    }

    // work of a step: strips of RPT interior rows of the interior column pairs
    // 1 .. PL-1 (tasks 0 .. nB-1, threads 0 ..), single edge pairs (rows 0 and
    // h-1, then the pairs 0 and PL of rows 1 .. h-2; threads nB ..), and the
    // 2w + 2h + 4 ring slots, fetched by the edge threads after their pairs
    const int PW = (w + 1) >> 1, PL = PW - 1;
    const int ncp = max(0, PL - 1);
    const int nrow = max(0, h - 2);
    const int nB = ncp * ((nrow + RPT - 1) / RPT);
    const int nEr = (h >= 2) ? 2 : 1;
    const int nEc = (PL > 0) ? 2 : 1;
    const int nA = nEr * PW + nrow * nEc;
    const int aFirst = (nB < kResThreads) ? nB : 0;
    const int aStride = kResThreads - aFirst;
    const int nslot = 2 * w + 2 * h + 4;

    const bool stall = tx == 0 && ty == 0 && *(volatile const int *)(err + 1) != 0;
    unsigned long long lim = *reinterpret_cast<volatile const unsigned long long *>(err + 2);
    if (lim == 0) lim = kDefaultWaitNs;

    // ring slot k: the neighbour word it copies (offset in xbuf of parity 0, or
    // -1 on the domain boundary, where the ring stays zero) and its place in a
    // state array
    auto slot_src = [&](int k, int &dst) -> long long {
        int nbx = tx, nby = ty, idx;
        if (k < w) {                                   // below the tile: the top row of (tx, ty-1)
            nby = ty - 1;
            idx = W + k;
            dst = k + 2;
        } else if (k < 2 * w) {                        // above: the bottom row of (tx, ty+1)
            nby = ty + 1;
            idx = k - w;
            dst = (h + 1) * SW + (k - w) + 2;
        } else if (k < 2 * w + h) {                    // left: the right column of (tx-1, ty)
            const int ly = k - 2 * w;
            nbx = tx - 1;
            idx = 2 * W + H + ly;
            dst = (ly + 1) * SW + 1;
        } else if (k < 2 * w + 2 * h) {                // right: the left column of (tx+1, ty)
            const int ly = k - 2 * w - h;
            nbx = tx + 1;
            idx = 2 * W + ly;
            dst = (ly + 1) * SW + w + 2;
        } else {                                       // corners, from the diagonal tiles' rows
            const int c = k - 2 * w - 2 * h;           // 0 (-1,-1), 1 (w,-1), 2 (-1,h), 3 (w,h)
            nbx = (c & 1) ? tx + 1 : tx - 1;
            nby = (c & 2) ? ty + 1 : ty - 1;
            idx = (c & 2) ? ((c & 1) ? 0 : W - 1) : ((c & 1) ? W : 2 * W - 1);
            dst = ((c & 2) ? h + 1 : 0) * SW + ((c & 1) ? w + 2 : 1);
        }
        if (nbx < 0 || nbx >= ntx || nby < 0 || nby >= nty) return -1;
        return (long long)(nby * ntx + nbx) * 2 * E + idx;
    };
    // copy ring slot k of state s into the state array U (bounded wait for its tag)
    auto fetch = [&](int k, int s, float *U) {
        int dst = 0;
        const long long src = slot_src(k, dst);
        if (src < 0) return;
        const unsigned long long *p = xbuf + src + (s & 1) * E;
        const unsigned want = (stall && s == 1) ? 0xffffffffu : (unsigned)(s + 1);
        unsigned long long v = ld_word(p);
        if ((unsigned)(v >> 32) != want) {
            const unsigned long long t0 = global_ns();
            for (int it = 1;; ++it) {
                v = ld_word(p);
                if ((unsigned)(v >> 32) == want) break;
                if ((it & 31) == 0 && *(volatile int *)err) {
                    s_abort = 1;
                    return;
                }
                if (global_ns() - t0 > lim) {
                    s_abort = 1;
                    atomicExch(err, 1);
                    return;
                }
            }
        }
        U[dst] = __uint_as_float((unsigned)v);
    };

    const Stencil2dCoef<float2> SC = stencil2d_coef2(C);
    const float2 n2 = pr(-2.f, -2.f);
    // u row ly (ring included) as the pairs (m, 0, p) = (u(lx-1+o), u(lx+o)), o = 0, 1, 2
    auto urow = [&](const float *P, int ly, int lx, float2 &m, float2 &z, float2 &p) {
        const float *q = P + (ly + 1) * SW + lx + 1;
        const float l = q[0];
        z = ld2(q + 1);
        const float r = q[3];
        m = pr(l, z.x);
        p = pr(z.y, r);
    };
    // cell row cy: k0 = cells left of the nodes (lx-1, lx), k1 = cells right of them
    auto krow = [&](int cy, int lx, float2 &k0, float2 &k1) {
        const float *q = K + (cy + 1) * SW + lx + 1;
        k1 = ld2(q + 1);
        k0 = pr(q[0], k1.x);
    };
    auto output = [&](int lx, int ly, float2 u, int fl, bool two) {
        const int64_t c = (y0 + ly) * L.nx + x0 + lx;
        if ((fl & 1) && slot->snap_part) {
            slot->snap_part[2 * c] = (double)u.x;
            if (two) slot->snap_part[2 * c + 2] = (double)u.y;
        }
        if ((fl & 2) && slot->final_part) {
            slot->final_part[2 * c] = (double)u.x;
            if (two) slot->final_part[2 * c + 2] = (double)u.y;
        }
    };

    __syncthreads();
    for (int j = 0; j < nsteps; ++j) {
        const float *cur = (j & 1) ? U1 : U0;          // u_j (ring filled)
        float *nxt = (j & 1) ? U0 : U1;                // u_{j-1}, becomes u_{j+1}
        const float2 abj = __ldg(ab + j);
        const float2 a2 = pr(abj.x, abj.x), nb2 = pr(-abj.y, -abj.y);
        const int fl = ((j + 1 == jim) ? 1 : 0) | ((j + 1 == jfin) ? 2 : 0);

        for (int t = tid; t < nB; t += kResThreads) {
            const int lx = 2 * (1 + t % ncp);
            const int r0 = 1 + (t / ncp) * RPT;
            const int r1 = min(r0 + RPT, h - 1);
            float2 umm, um0, ump, u0m, u00, u0p, k00, k01;
            urow(cur, r0 - 1, lx, umm, um0, ump);
            urow(cur, r0, lx, u0m, u00, u0p);
            float2 pm = vadd(umm, ump), p0 = vadd(u0m, u0p);
            krow(r0 - 1, lx, k00, k01);
            float2 hk0 = vadd(k00, k01);
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int ly = r0 + i;
                if (ly >= r1) break;
                float2 upm, up0, upp, k10, k11;
                urow(cur, ly + 1, lx, upm, up0, upp);
                krow(ly, lx, k10, k11);
                const float2 pp = vadd(upm, upp);
                const float2 hk1 = vadd(k10, k11);
                const float2 acc = stencil2d(SC, umm, um0, ump, u0m, u00, u0p, upm, up0, upp, k00,
                                             k01, k10, k11, pm, p0, pp, hk0, hk1);
                const int ni = ly * W + lx, si = (ly + 1) * SW + lx + 2;
                const float2 ag = vfma(a2, ld2(FR + ni), vfma(nb2, ld2(FI + ni), acc));
                const float2 uprev = ld2(nxt + si);
                const float2 unew = vfma(ld2(D + ni), vfma(n2, uprev, ag), uprev);
                st2(nxt + si, unew);
                if (fl) output(lx, ly, unew, fl, true);
                umm = u0m; um0 = u00; ump = u0p; pm = p0;
                u0m = upm; u00 = up0; u0p = upp; p0 = pp;
                k00 = k10; k01 = k11; hk0 = hk1;
            }
        }
        if (tid >= aFirst) {
            const unsigned tag = (unsigned)(j + 2);
            unsigned long long *pub = mine + ((j + 1) & 1) * E;
            auto publish = [&](int lx, int ly, float v) {
                if (ly == 0) st_word(pub + lx, v, tag);
                if (ly == h - 1) st_word(pub + W + lx, v, tag);
                if (lx == 0) st_word(pub + 2 * W + ly, v, tag);
                if (lx == w - 1) st_word(pub + 2 * W + H + ly, v, tag);
            };
            for (int a = tid - aFirst; a < nA; a += aStride) {
                int ly, p;
                if (a < nEr * PW) {
                    ly = (a < PW) ? 0 : h - 1;
                    p = (a < PW) ? a : a - PW;
                } else {
                    const int b = a - nEr * PW;
                    ly = 1 + b / nEc;
                    p = (b % nEc) ? PL : 0;
                }
                const int lx = 2 * p;
                float2 umm, um0, ump, u0m, u00, u0p, upm, up0, upp, k00, k01, k10, k11;
                urow(cur, ly - 1, lx, umm, um0, ump);
                urow(cur, ly, lx, u0m, u00, u0p);
                urow(cur, ly + 1, lx, upm, up0, upp);
                krow(ly - 1, lx, k00, k01);
                krow(ly, lx, k10, k11);
                const float2 acc =
                    stencil2d(SC, umm, um0, ump, u0m, u00, u0p, upm, up0, upp, k00, k01, k10, k11,
                              vadd(umm, ump), vadd(u0m, u0p), vadd(upm, upp), vadd(k00, k01),
                              vadd(k10, k11));
                const int ni = ly * W + lx, si = (ly + 1) * SW + lx + 2;
                const float2 ag = vfma(a2, ld2(FR + ni), vfma(nb2, ld2(FI + ni), acc));
                const float2 uprev = ld2(nxt + si);
                const float2 unew = vfma(ld2(D + ni), vfma(n2, uprev, ag), uprev);
                const bool two = lx + 1 < w;                // the second node is in the tile
                if (two) st2(nxt + si, unew);
                else nxt[si] = unew.x;
                publish(lx, ly, unew.x);
                if (two) publish(lx + 1, ly, unew.y);
                if (fl) output(lx, ly, unew, fl, two);
            }
            if (j + 1 < nsteps)
                for (int k = tid - aFirst; k < nslot; k += aStride) fetch(k, j + 1, nxt);
        }
        __syncthreads();
        if (s_abort) break;
    }
}

template <int RPT>
bool set_smem_attr(size_t smem)
{
    return cudaFuncSetAttribute(res2d_kernel<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem) == cudaSuccess;
}

// edge and interior tasks of a full W x H tile with RPT rows per strip
int res2d_tasks(int W, int H, int rpt)
{
    const int PW = (W + 1) / 2, PL = PW - 1;
    const int nrow = std::max(0, H - 2);
    const int nB = std::max(0, PL - 1) * ((nrow + rpt - 1) / rpt);
    const int nA = ((H >= 2) ? 2 : 1) * PW + nrow * ((PL > 0) ? 2 : 1);
    return nA + nB;
}

}  // namespace

bool res2d_plan(const Layout &L, Res2dPlan *out)
{
    if (L.d != 2 || L.nx < 1 || L.ny < 1) return false;
    int dev = 0, nsm = 0, coop = 0, maxsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (!coop || nsm < 1) return false;
    // the tiling with the smallest largest tile (then the shortest edges) that
    // fits one tile per CTA, one CTA per SM
    Res2dPlan best;
    long long best_area = -1, best_edge = 0;
    for (int a = 1; a <= nsm; ++a) {
        long long W = (L.nx + a - 1) / a;
        W += W & 1;
        const long long ntx = (L.nx + W - 1) / W;
        const long long tiles_y = nsm / ntx;
        if (tiles_y < 1) break;
        const long long H = (L.ny + tiles_y - 1) / tiles_y;
        const long long nty = (L.ny + H - 1) / H;
        if (W > 4096 || H > 4096) continue;
        const size_t smem = res2d_floats((int)W, (int)H) * sizeof(float);
        if (smem > (size_t)maxsm) continue;
        const long long area = W * H, edge = W + H;
        if (best_area < 0 || area < best_area || (area == best_area && edge < best_edge)) {
            best_area = area;
            best_edge = edge;
            best.W = (int)W;
            best.H = (int)H;
            best.ntx = (int)ntx;
            best.nty = (int)nty;
            best.smem = smem;
        }
    }
    if (best_area < 0) return false;
    best.rpt = 16;
    for (int r : {4, 8, 12, 16})
        if (res2d_tasks(best.W, best.H, r) <= kResThreads) {
            best.rpt = r;
            break;
        }
    const bool attr = best.rpt == 4    ? set_smem_attr<4>(best.smem)
                      : best.rpt == 8  ? set_smem_attr<8>(best.smem)
                      : best.rpt == 12 ? set_smem_attr<12>(best.smem)
                                       : set_smem_attr<16>(best.smem);
    int occ = 0;
    const cudaError_t oe =
        best.rpt == 4    ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, res2d_kernel<4>, kResThreads, best.smem)
        : best.rpt == 8  ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, res2d_kernel<8>, kResThreads, best.smem)
        : best.rpt == 12 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, res2d_kernel<12>, kResThreads, best.smem)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, res2d_kernel<16>, kResThreads, best.smem);
    if (!attr || oe != cudaSuccess || occ < 1 || (long long)best.ntx * best.nty > (long long)occ * nsm) {
        (void)cudaGetLastError();
        return false;
    }
    best.xwords = (size_t)best.ntx * best.nty * 2 * (2 * (size_t)best.W + 2 * (size_t)best.H);
    *out = best;
    return true;
}

void launch_res2d(const Res2dPlan &p, const float *kap, const float *dco, const float *fre,
                  const float *fim, const Layout &L, const StepCoef<float> &C, const float2 *ab,
                  int nsteps, int jim, int jfin, const OutSlot *slot, unsigned long long *xbuf,
                  int *err, cudaStream_t s)
{
    (void)cudaMemsetAsync(xbuf, 0, p.xwords * sizeof(unsigned long long), s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.ntx, (unsigned)p.nty);
    cfg.blockDim = dim3(kResThreads);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define HTD_RES2D_LAUNCH(R)                                                                     \
    (void)cudaLaunchKernelEx(&cfg, res2d_kernel<R>, kap, dco, fre, fim, L, C, ab, nsteps, jim, \
                             jfin, slot, xbuf, err, p.W, p.H)
    switch (p.rpt) {
        case 4: HTD_RES2D_LAUNCH(4); break;
        case 8: HTD_RES2D_LAUNCH(8); break;
        case 12: HTD_RES2D_LAUNCH(12); break;
        default: HTD_RES2D_LAUNCH(16); break;
    }
#undef HTD_RES2D_LAUNCH
    ++g_launches;
}

}  // namespace htd
