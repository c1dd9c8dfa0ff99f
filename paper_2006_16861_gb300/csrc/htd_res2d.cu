// Resident-grid 2-D recurrence (FP32 or FP64, node pairs): the whole grid
// stays in shared memory, spread over the SMs, for all T n_P steps of a run.
//
// One cooperative launch runs a whole preconditioner run (Def. of I_acd with
// Table 1's windowed forcing and read-out).  The grid is cut into ntx x nty
// tiles of W x H nodes, one CTA per tile and at most one CTA per SM, every CTA
// resident at once.  A CTA loads its tile's q*kappa cells, d and forcing once,
// keeps both recurrence states in shared memory with a one-node ring around
// the tile, and in every step
//  - computes the new state of its edge nodes first (one edge pair per
//    thread) and publishes each edge value to a global exchange buffer as
//    tagged 64-bit words (tag = index of the state + 1; an FP32 value in one
//    word with its bits, an FP64 value in two words, one per 32-bit half; one
//    buffer per state parity);
//  - computes its interior nodes in row strips with a 3 x 3 register window;
//    the strip threads also read the neighbours' edge words of the new state
//    into the ring: each read is issued two rows into the thread's strip and
//    its tags checked after the strip, re-reading until they are the expected
//    ones (bounded by the handle's wait limit);
//  - passes one CTA barrier.
// Each exchanged word carries its own tag and moves as one 64-bit access, so
// no fence has to order data before a flag.  A CTA cannot run more than one
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
#include <type_traits>

#include "htd_internal.h"

namespace htd {

namespace {

// threads per CTA: 768 for FP32 (80 registers each), 512 for FP64 (its
// register windows are twice as wide)
template <typename T>
__host__ __device__ constexpr int res_threads()
{
    return sizeof(T) == 8 ? 512 : 768;
}

// A node pair (lx, lx + 1) as one value: float2 for the FP32 recurrence
// (paired FP32 instructions), DPair for FP64 (two scalar FP64 operations, each
// lane rounded like the one-step kernel's scalar).
struct __align__(16) DPair {
    double x, y;
};
// (the FP32 and scalar overloads of the enclosing namespace stay visible)
using htd::vadd;
using htd::vfma;
using htd::vmul;
__device__ __forceinline__ DPair vadd(DPair a, DPair b) { return {__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)}; }
__device__ __forceinline__ DPair vmul(DPair a, DPair b) { return {__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)}; }
__device__ __forceinline__ DPair vfma(DPair a, DPair b, DPair c)
{
    return {__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y)};
}

template <typename T>
struct PairOf;
template <>
struct PairOf<float> {
    typedef float2 V;
    __device__ static V make(float a, float b) { return make_float2(a, b); }
};
template <>
struct PairOf<double> {
    typedef DPair V;
    __device__ static V make(double a, double b) { return {a, b}; }
};

template <typename T>
__device__ __forceinline__ typename PairOf<T>::V ld2(const T *p)
{
    return *reinterpret_cast<const typename PairOf<T>::V *>(p);
}

template <typename T>
__device__ __forceinline__ void st2(T *p, typename PairOf<T>::V v)
{
    *reinterpret_cast<typename PairOf<T>::V *>(p) = v;
}

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

__device__ __forceinline__ void st_word(unsigned long long *p, unsigned bits, unsigned tag)
{
    const unsigned long long w = ((unsigned long long)tag << 32) | bits;
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

// An exchanged value as tagged words: an FP32 value in one word, an FP64 value
// in two (low and high halves, each with the tag), valid when every tag is the
// expected one.
template <typename T>
struct Xword;
template <>
struct Xword<float> {
    static constexpr int kPer = 1;
    struct Raw {
        unsigned long long w;
    };
    __device__ static void put(unsigned long long *p, float v, unsigned tag)
    {
        st_word(p, __float_as_uint(v), tag);
    }
    __device__ static Raw get(const unsigned long long *p) { return {ld_word(p)}; }
    __device__ static bool ok(const Raw &r, unsigned want) { return (unsigned)(r.w >> 32) == want; }
    __device__ static float value(const Raw &r) { return __uint_as_float((unsigned)r.w); }
};
template <>
struct Xword<double> {
    static constexpr int kPer = 2;
    struct Raw {
        unsigned long long lo, hi;
    };
    __device__ static void put(unsigned long long *p, double v, unsigned tag)
    {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        st_word(p, (unsigned)b, tag);
        st_word(p + 1, (unsigned)(b >> 32), tag);
    }
    __device__ static Raw get(const unsigned long long *p) { return {ld_word(p), ld_word(p + 1)}; }
    __device__ static bool ok(const Raw &r, unsigned want)
    {
        return (unsigned)(r.lo >> 32) == want && (unsigned)(r.hi >> 32) == want;
    }
    __device__ static double value(const Raw &r)
    {
        return __longlong_as_double((long long)((r.hi << 32) | (r.lo & 0xffffffffull)));
    }
};

// the step coefficients broadcast to node pairs
__device__ __forceinline__ Stencil2dCoef<float2> pair_coef(const StepCoef<float> &C)
{
    return stencil2d_coef2(C);
}

__device__ __forceinline__ Stencil2dCoef<DPair> pair_coef(const StepCoef<double> &C)
{
    auto b = [](double x) { return DPair{x, x}; };
    return {b(C.c0), b(C.mt[0]), b(C.mt[1]), b(C.mt[2]), b(-C.cs[1]), b(-C.cs[2])};
}

// row strides of the shared-memory arrays the kernel is built for (8 banks of
// 4 bytes apart from row to row for FP32); a tile of width W uses the smallest
// one >= W + 4
constexpr int kStrides[] = {72, 136};

__host__ __device__ constexpr size_t res2d_elems(int SW, int H)
{
    return 6 * (size_t)(H + 2) * SW;
}

// Shared memory: six arrays of (H + 2) rows of SW elements of T -- the states
// U0, U1, the cells K, and d, Re F, Im F -- with node (lx, ly) of the tile at
// row ly + 1, column lx + 2 of each (so the pair (lx, lx + 1), lx even, is
// aligned for one vector access, and one offset addresses a node in all six),
// the state ring at rows 0 and h + 1 and columns 1 and w + 2, and cell
// (cx, cy) (its lower corner node) at the place of node (cx, cy).  Exchange
// buffer of a tile and parity: E = 2W + 2H values (X::kPer words each) --
// bottom row [0, W), top row [W, 2W), left column [2W, 2W + H), right column
// [2W + H, 2W + 2H).
template <typename T, int RPT, int SW>
__global__ void __launch_bounds__(res_threads<T>(), 1)
res2d_kernel(const T *__restrict__ kap, const T *__restrict__ dco, const T *__restrict__ fre,
             const T *__restrict__ fim, Layout L, StepCoef<T> C,
             const typename PairOf<T>::V *__restrict__ ab, int nsteps, int jim, int jfin,
             const OutSlot *__restrict__ slot, unsigned long long *__restrict__ xbuf,
             int *__restrict__ err, int W, int H, Res2dProj<T> P)
{
    typedef typename PairOf<T>::V V;
    typedef Xword<T> X;
    constexpr int NT = res_threads<T>();
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    __shared__ int s_abort;
    auto pr = [](T a, T b) { return PairOf<T>::make(a, b); };
    const int tid = threadIdx.x;
    const int tx = blockIdx.x, ty = blockIdx.y;
    const int ntx = gridDim.x, nty = gridDim.y;
    const int64_t x0 = (int64_t)tx * W, y0 = (int64_t)ty * H;
    const int w = (int)min((int64_t)W, L.nx - x0);
    const int h = (int)min((int64_t)H, L.ny - y0);
    const int NA = (H + 2) * SW;
    T *U0 = sm, *U1 = sm + NA, *K = sm + 2 * NA;
    T *D = sm + 3 * NA, *FR = sm + 4 * NA, *FI = sm + 5 * NA;
    const int EW = (2 * W + 2 * H) * X::kPer;          // exchange words per tile and parity

    if (tid == 0) s_abort = 0;
    for (int i = tid; i < NA; i += NT) {
        const int ly = i / SW - 1, lx = i % SW - 2;
        T k = 0, dv = 0, fr = 0, fi = 0;
        if (lx >= -1 && lx < w && ly >= -1 && ly < h) {
            const int64_t g = (y0 + ly + 1) * L.pitch + L.xl + x0 + lx;
            k = kap[g];                                // cell (lx, ly)
            if (lx >= 0 && ly >= 0) {
                dv = dco[g];
                fr = fre[g];
                fi = fim[g];
            }
        }
        U0[i] = 0.f;
        U1[i] = 0.f;
        K[i] = k;
        D[i] = dv;
        FR[i] = fr;
        FI[i] = fi;
    }

    // Work of a step, per thread in this order: (1) an edge pair -- rows 0 and
    // h-1, then the pairs 0 and PL of rows 1 .. h-2 -- dealt one per thread
    // from the last thread down, so that threads without interior work take
    // them first (several edge pairs on one thread publish the later ones too
    // late for the neighbours); each new edge value is published at once; (2) one strip of up to RPT interior
    // rows of an interior column pair 1 .. PL-1 (strip t on thread t); (3) the
    // ring slot of the next state (slot k on thread k): the read of the
    // neighbour's word is issued two rows into the thread's strip and its tag
    // checked after the strip, so that the exchange overlaps the interior
    // work; the word is read again only if the neighbour had not published it.
    // The geometry of all three is the same in every step.
    const int PW = (w + 1) >> 1, PL = PW - 1;
    const int ncp = max(0, PL - 1);
    const int nrow = max(0, h - 2);
    const int nS = ncp * ((nrow + RPT - 1) / RPT);
    const int nEr = (h >= 2) ? 2 : 1;
    const int nEc = (PL > 0) ? 2 : 1;
    const int nA = nEr * PW + nrow * nEc;
    const int nslot = 2 * w + 2 * h + 4;
    // (1) the edge pair of task a as (node offset, lx, ly)
    auto edge_of = [&](int a, int &lx, int &ly) {
        int p;
        if (a < nEr * PW) {
            ly = (a < PW) ? 0 : h - 1;
            p = (a < PW) ? a : a - PW;
        } else {
            const int b = a - nEr * PW;
            ly = 1 + b / nEc;
            p = (b % nEc) ? PL : 0;
        }
        lx = 2 * p;
    };
    const int ea = NT - 1 - tid;              // this thread's first edge task
    int e_lx = 0, e_ly = 0;
    if (ea < nA) edge_of(ea, e_lx, e_ly);
    // (2) strip t: column pair, first row, rows
    auto strip_of = [&](int t, int &lx, int &r0, int &nr) -> bool {
        lx = 2 * (1 + t % ncp);
        r0 = 1 + (t / ncp) * RPT;
        nr = min(RPT, h - 1 - r0);
        return true;
    };
    int s_lx = 0, s_r0 = 1, s_nr = 0;
    const bool has_strip = tid < nS && strip_of(tid, s_lx, s_r0, s_nr);
    // (3) the ring slot: the neighbour's word (offset in xbuf for parity 0, or
    // -1 on the domain boundary, where the ring stays zero) and its place in a
    // state array
    auto slot_of = [&](int k, int &dst) -> int {
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
        return (nby * ntx + nbx) * 2 * EW + idx * X::kPer;
    };
    int r_dst = 0;
    const int r_src = (tid < nslot) ? slot_of(tid, r_dst) : -1;

    // store slot value v (read from p) of state s into U at dst, reading it again
    // until its words carry the tag of state s (bounded by the handle's limit;
    // with the stall test the first wait of CTA (0, 0) expects a tag no word has)
    auto complete = [&](const unsigned long long *p, typename X::Raw v, int s, int dst, T *U) {
        unsigned want = (unsigned)(s + 1);
        if (s == 1 && tx == 0 && ty == 0 && *(volatile const int *)(err + 1) != 0)
            want = 0xffffffffu;
        if (!X::ok(v, want)) {
            unsigned long long lim = *reinterpret_cast<volatile const unsigned long long *>(err + 2);
            if (lim == 0) lim = kDefaultWaitNs;
            const unsigned long long t0 = global_ns();
            for (int it = 1;; ++it) {
                v = X::get(p);
                if (X::ok(v, want)) break;
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
        U[dst] = X::value(v);
    };

    const Stencil2dCoef<V> SC = pair_coef(C);
    const V n2 = pr(T(-2), T(-2));
    // u row at q (the node lx - 1 of the row) as the pairs (m, 0, p) =
    // (u(lx-1+o), u(lx+o)), o = 0, 1, 2
    auto urow = [&](const T *q, V &m, V &z, V &p) {
        const T l = q[0];
        z = ld2(q + 1);
        const T r = q[3];
        m = pr(l, z.x);
        p = pr(z.y, r);
    };
    // cells at q (the cell lx - 1 of a cell row): k0 = cells left of the nodes
    // (lx-1, lx), k1 = cells right of them
    auto krow = [&](const T *q, V &k0, V &k1) {
        k1 = ld2(q + 1);
        k0 = pr(q[0], k1.x);
    };
    auto output = [&](int lx, int ly, V u, int fl, bool two) {
        const int64_t c = ((int64_t)blockIdx.y * H + ly) * L.nx + (int64_t)blockIdx.x * W + lx;
        if ((fl & 1) && slot->snap_part) {
            slot->snap_part[2 * c] = (double)u.x;
            if (two) slot->snap_part[2 * c + 2] = (double)u.y;
        }
        if ((fl & 2) && slot->final_part) {
            slot->final_part[2 * c] = (double)u.x;
            if (two) slot->final_part[2 * c + 2] = (double)u.y;
        }
    };
    // the new state of the pair at node offset o (row ly + 1, column lx + 2)
    // from its stencil sum
    auto update = [&](int o, V acc, V a2, V nb2, T *nxt) -> V {
        const V ag = vfma(a2, ld2(FR + o), vfma(nb2, ld2(FI + o), acc));
        const V uprev = ld2(nxt + o);
        return vfma(ld2(D + o), vfma(n2, uprev, ag), uprev);
    };
    // nr <= RPT interior rows r0 .. r0+nr-1 of the column pair lx; the read of
    // the ring word at rp (if any) is issued before the third row
    // (kFull: nr == RPT, so the unrolled rows need no test; kOut: a step with
    // output flags)
    auto strip = [&](int lx, int r0, int nr, const T *cur, T *nxt, V a2, V nb2, int fl,
                     const unsigned long long *rp, typename X::Raw &rv, bool &issued,
                     auto full_tag, auto out_tag) {
        constexpr bool kFull = decltype(full_tag)::value, kOut = decltype(out_tag)::value;
        const int o0 = r0 * SW + lx + 1;               // node (lx - 1, r0 - 1)
        const T *qc = cur + o0, *qk = K + o0;
        V umm, um0, ump, u0m, u00, u0p, k00, k01;
        urow(qc, umm, um0, ump);
        urow(qc + SW, u0m, u00, u0p);
        V pm = vadd(umm, ump), p0 = vadd(u0m, u0p);
        krow(qk, k00, k01);
        V hk0 = vadd(k00, k01);
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            if (!kFull && i >= nr) break;
            if (i == 2 && rp) {
                rv = X::get(rp);
                issued = true;
            }
            V upm, up0, upp, k10, k11;
            urow(qc + (i + 2) * SW, upm, up0, upp);
            krow(qk + (i + 1) * SW, k10, k11);
            const V pp = vadd(upm, upp);
            const V hk1 = vadd(k10, k11);
            const V acc = stencil2d(SC, umm, um0, ump, u0m, u00, u0p, upm, up0, upp, k00, k01,
                                         k10, k11, pm, p0, pp, hk0, hk1);
            const int o = o0 + (i + 1) * SW + 1;       // node (lx, r0 + i)
            const V unew = update(o, acc, a2, nb2, nxt);
            st2(nxt + o, unew);
            if (kOut) output(lx, r0 + i, unew, fl, true);
            umm = u0m; um0 = u00; ump = u0p; pm = p0;
            u0m = upm; u00 = up0; u0p = upp; p0 = pp;
            k00 = k10; k01 = k11; hk0 = hk1;
        }
    };

    __syncthreads();
    for (int j = 0; j < nsteps; ++j) {
        const T *cur = (j & 1) ? U1 : U0;              // u_j (ring filled)
        T *nxt = (j & 1) ? U0 : U1;                    // u_{j-1}, becomes u_{j+1}
        const V abj = ab[j];
        const V a2 = pr(abj.x, abj.x), nb2 = pr(-abj.y, -abj.y);
        const int fl = ((j + 1 == jim) ? 1 : 0) | ((j + 1 == jfin) ? 2 : 0);
        const bool more = j + 1 < nsteps;

        // (1) edge pairs, published as they are computed
        if (ea < nA) {
            const unsigned tag = (unsigned)(j + 2);
            unsigned long long *pub = xbuf + (size_t)((ty * ntx + tx) * 2 + ((j + 1) & 1)) * EW;
            auto publish = [&](int lx, int ly, T v) {
                if (ly == 0) X::put(pub + X::kPer * lx, v, tag);
                if (ly == h - 1) X::put(pub + X::kPer * (W + lx), v, tag);
                if (lx == 0) X::put(pub + X::kPer * (2 * W + ly), v, tag);
                if (lx == w - 1) X::put(pub + X::kPer * (2 * W + H + ly), v, tag);
            };
            for (int a = ea; a < nA; a += NT) {
                int lx = e_lx, ly = e_ly;
                if (a != ea) edge_of(a, lx, ly);
                const int o = (ly + 1) * SW + lx + 2;
                V umm, um0, ump, u0m, u00, u0p, upm, up0, upp, k00, k01, k10, k11;
                urow(cur + o - SW - 1, umm, um0, ump);
                urow(cur + o - 1, u0m, u00, u0p);
                urow(cur + o + SW - 1, upm, up0, upp);
                krow(K + o - SW - 1, k00, k01);
                krow(K + o - 1, k10, k11);
                const V acc =
                    stencil2d(SC, umm, um0, ump, u0m, u00, u0p, upm, up0, upp, k00, k01, k10, k11,
                              vadd(umm, ump), vadd(u0m, u0p), vadd(upm, upp), vadd(k00, k01),
                              vadd(k10, k11));
                const V unew = update(o, acc, a2, nb2, nxt);
                const bool two = lx + 1 < w;                // the second node is in the tile
                if (two) st2(nxt + o, unew);
                else nxt[o] = unew.x;
                publish(lx, ly, unew.x);
                if (two) publish(lx + 1, ly, unew.y);
                if (fl) output(lx, ly, unew, fl, two);
            }
        }

        // (2) the interior strip, with the read of this thread's ring slot
        const unsigned long long *rp =
            (more && r_src >= 0) ? xbuf + r_src + ((j + 1) & 1) * EW : nullptr;
        typename X::Raw rv{};
        bool issued = false;
        using T_ = std::true_type;
        using F_ = std::false_type;
        if (has_strip) {
            if (s_nr == RPT) {
                if (fl) strip(s_lx, s_r0, s_nr, cur, nxt, a2, nb2, fl, rp, rv, issued, T_{}, T_{});
                else strip(s_lx, s_r0, s_nr, cur, nxt, a2, nb2, fl, rp, rv, issued, T_{}, F_{});
            } else {
                strip(s_lx, s_r0, s_nr, cur, nxt, a2, nb2, fl, rp, rv, issued, F_{}, T_{});
            }
        }
        for (int t = tid + NT; t < nS; t += NT) {
            int lx, r0, nr;
            if (strip_of(t, lx, r0, nr))
                strip(lx, r0, nr, cur, nxt, a2, nb2, fl, nullptr, rv, issued, F_{}, T_{});
        }

        // (3) the ring of u_{j+1}
        if (rp) complete(rp, issued ? rv : X::get(rp), j + 1, r_dst, nxt);
        if (more)
            for (int k = tid + NT; k < nslot; k += NT) {
                int dst = 0;
                const int src = slot_of(k, dst);
                if (src < 0) continue;
                const unsigned long long *p = xbuf + src + ((j + 1) & 1) * EW;
                complete(p, X::get(p), j + 1, dst, nxt);
            }
        __syncthreads();
        if (s_abort) break;
        // projection read-out: the compensated accumulation of u_{j+1} (complete
        // in nxt, which the next step only reads) into the sums and
        // compensations (re, im), as the separate accumulation kernel does it,
        // the tile's nodes in compact order
        if (j >= P.j_acc) {
            const int k = (j + 1) % P.nP;
            const T wc = P.w[2 * k], ws = P.w[2 * k + 1];
            T *a = P.acc;
            for (int i = tid; i < w * h; i += NT) {
                const int ly = i / w, lx = i - ly * w;
                const int64_t c = ((int64_t)blockIdx.y * H + ly) * L.nx +
                                  (int64_t)blockIdx.x * W + lx;
                const T v = nxt[(ly + 1) * SW + lx + 2];
                T sr = a[c], si = a[P.N + c], cr = a[2 * P.N + c], ci = a[3 * P.N + c];
                const T yr = wc * v - cr, yi = ws * v - ci;
                const T tr = sr + yr, ti = si + yi;
                a[2 * P.N + c] = (tr - sr) - yr;
                a[3 * P.N + c] = (ti - si) - yi;
                a[c] = tr;
                a[P.N + c] = ti;
            }
        }
    }
}

// Rows per strip a plan may choose: FP32 3, 5 or 8; FP64 also 1 -- its
// long-latency FP64 pipe makes a thread's chain of dependent rows, not the
// register window's saved loads, what sets the step time on small tiles
// (one-row strips in FP32 measured no faster at 101^2).
constexpr int kRpts[] = {1, 3, 5, 8};

template <typename T>
bool rpt_allowed(int r)
{
    return r != 1 || sizeof(T) == 8;
}

// fn(the kernel for precision T, RPT rows per strip, row stride SW)
template <typename T, typename Fn>
void with_kernel(int rpt, int sw, Fn &&fn)
{
    if (sw == 72) {
        if (rpt == 1) fn(res2d_kernel<T, 1, 72>);
        else if (rpt == 3) fn(res2d_kernel<T, 3, 72>);
        else if (rpt == 5) fn(res2d_kernel<T, 5, 72>);
        else fn(res2d_kernel<T, 8, 72>);
    } else {
        if (rpt == 1) fn(res2d_kernel<T, 1, 136>);
        else if (rpt == 3) fn(res2d_kernel<T, 3, 136>);
        else if (rpt == 5) fn(res2d_kernel<T, 5, 136>);
        else fn(res2d_kernel<T, 8, 136>);
    }
}

// Rows of work of the busiest thread of a full W x H tile with RPT rows per
// strip (an edge pair counted as two rows: it has no register window), or -1
// if there are more strips than threads.
int res2d_load(int W, int H, int rpt, int NT)
{
    const int PW = (W + 1) / 2, PL = PW - 1;
    const int nrow = std::max(0, H - 2);
    const int nS = std::max(0, PL - 1) * ((nrow + rpt - 1) / rpt);
    const int nA = ((H >= 2) ? 2 : 1) * PW + nrow * ((PL > 0) ? 2 : 1);
    if (nS > NT) return -1;
    const int edges = (nA + NT - 1) / NT;                       // edge pairs per thread
    return std::min(rpt, nrow) + 2 * (nS + nA > NT ? edges : 0);
}

template <typename T>
bool plan_impl(const Layout &L, Res2dPlan *out)
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
    // the limit is a property of the kernel, shared by every handle: raise it
    // to what the device allows beside the kernel's static shared memory,
    // rather than to this plan's size (a smaller plan made later must not
    // shrink it under an earlier handle's launches)
    int avail = maxsm;
    bool attr_ok = true;
    for (int sw : kStrides)
        for (int r : kRpts) {
            if (!rpt_allowed<T>(r)) continue;
            with_kernel<T>(r, sw, [&](auto kern) {
                cudaFuncAttributes fa;
                if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
                    attr_ok = false;
                    return;
                }
                const int dyn = maxsm - (int)fa.sharedSizeBytes;
                avail = std::min(avail, dyn);
                attr_ok = attr_ok && dyn > 0 &&
                          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               dyn) == cudaSuccess;
            });
        }
    if (!attr_ok) {
        (void)cudaGetLastError();
        return false;
    }
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
        int sw = 0;
        for (int s : kStrides)
            if (sw == 0 && W + 4 <= s) sw = s;
        if (sw == 0 || H > 4096) continue;
        const size_t smem = res2d_elems(sw, (int)H) * sizeof(T);
        if (smem > (size_t)avail) continue;
        const long long area = W * H, edge = W + H;
        if (best_area < 0 || area < best_area || (area == best_area && edge < best_edge)) {
            best_area = area;
            best_edge = edge;
            best.W = (int)W;
            best.H = (int)H;
            best.sw = sw;
            best.ntx = (int)ntx;
            best.nty = (int)nty;
            best.smem = smem;
        }
    }
    if (best_area < 0) return false;
    best.rpt = kRpts[sizeof(kRpts) / sizeof(kRpts[0]) - 1];
    int best_load = -1;
    for (int r : kRpts) {
        if (!rpt_allowed<T>(r)) continue;
        const int ld = res2d_load(best.W, best.H, r, res_threads<T>());
        if (ld >= 0 && (best_load < 0 || ld < best_load)) {
            best_load = ld;
            best.rpt = r;
        }
    }
    int occ = 0;
    cudaError_t oe = cudaSuccess;
    with_kernel<T>(best.rpt, best.sw, [&](auto kern) {
        oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, res_threads<T>(),
                                                           best.smem);
    });
    if (oe != cudaSuccess || occ < 1 || (long long)best.ntx * best.nty > (long long)occ * nsm) {
        (void)cudaGetLastError();
        return false;
    }
    best.xwords = (size_t)best.ntx * best.nty * 2 * (2 * (size_t)best.W + 2 * (size_t)best.H) *
                  Xword<T>::kPer;
    *out = best;
    return true;
}

}  // namespace

template <typename T>
bool res2d_plan(const Layout &L, Res2dPlan *p)
{
    return plan_impl<T>(L, p);
}

template <typename T>
void launch_res2d(const Res2dPlan &p, const T *kap, const T *dco, const T *fre, const T *fim,
                  const Layout &L, const StepCoef<T> &C, const T *ab, int nsteps, int jim,
                  int jfin, const OutSlot *slot, unsigned long long *xbuf, int *err,
                  cudaStream_t s, const Res2dProj<T> &P)
{
    (void)cudaMemsetAsync(xbuf, 0, p.xwords * sizeof(unsigned long long), s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.ntx, (unsigned)p.nty);
    cfg.blockDim = dim3(res_threads<T>());
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const auto *abv = reinterpret_cast<const typename PairOf<T>::V *>(ab);
    with_kernel<T>(p.rpt, p.sw, [&](auto kern) {
        (void)cudaLaunchKernelEx(&cfg, kern, kap, dco, fre, fim, L, C, abv, nsteps, jim, jfin,
                                 slot, xbuf, err, p.W, p.H, P);
    });
    ++g_launches;
}

template bool res2d_plan<float>(const Layout &, Res2dPlan *);
template bool res2d_plan<double>(const Layout &, Res2dPlan *);
template void launch_res2d<float>(const Res2dPlan &, const float *, const float *, const float *,
                                  const float *, const Layout &, const StepCoef<float> &,
                                  const float *, int, int, int, const OutSlot *,
                                  unsigned long long *, int *, cudaStream_t,
                                  const Res2dProj<float> &);
template void launch_res2d<double>(const Res2dPlan &, const double *, const double *,
                                   const double *, const double *, const Layout &,
                                   const StepCoef<double> &, const double *, int, int, int,
                                   const OutSlot *, unsigned long long *, int *, cudaStream_t,
                                   const Res2dProj<double> &);

}  // namespace htd
