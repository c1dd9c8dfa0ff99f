// CUDA kernels of the time-domain Helmholtz preconditioner (sm_103a).
//
//  step2d / step3d   one step of the frequency-adapted leapfrog recurrence
//                    I_acd (Def. of I_acd) with the windowed forcing of
//                    Table 1 fused in, in place over u_{j-1}, and the
//                    snapshot / final-state write of Table 1 fused in.
//  split             complex128 right-hand side -> Re/Im planes (Table 1 uses
//                    Re F and Im F every step).
//  apply_H           true operator H X (or F - H X), complex128, FP64.
//  dots / reduce     block dot products conj(V_k) . w with warp shuffles,
//                    two-pass fixed-order reduction (deterministic).
//  sub/add_combination, scale   Krylov vector updates.
//
// Operator (App. A cell form, h^2-scaled): for node beta and offset
// o in {-1,0,1}^d with Hamming weight s = |o|,
//   h^2 (Re H u)_beta = sum_o u_{beta+o} [ 2^{d-s} S_s - M_s * sum of kappa over
//                       the 2^{d-s} cells that contain both beta and beta+o ],
// kappa = (h k_cell)^2, S_s / M_s the stiffness / mass weights of the cell
// kernel at Hamming distance s.  One step of I_acd with
// K = (dt^2/alpha)(Re H + omega^2), L/2 = ell, d = 1/(1+ell):
//   u_{j+1} = d ((2 - K) u_j + g_j - 2 u_{j-1}) + u_{j-1},
//   g_j = a_j Re F - b_j Im F,
// where (2 - K) u_j = c0 u - sum_{o != 0} cs_s u_{beta+o}
//                     + sum_o M_s (sum of q kappa over the cells) u_{beta+o},
// q = dt^2 / (alpha h^2), c0 = 2 - (dt^2/alpha) omega^2 - q 2^d S_0,
// cs_s = q 2^{d-s} S_s; the stored per-cell coefficient is q * kappa.
#include <cuda_runtime.h>
#include <algorithm>

#include "htd_internal.h"

namespace htd {

long long g_launches = 0;

// ---------------------------------------------------------------------------
// recurrence step
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(256)
step2d_kernel(const T *__restrict__ u, T *__restrict__ um, const T *__restrict__ kap,
              const T *__restrict__ dco, const T *__restrict__ fre, const T *__restrict__ fim,
              Layout L, StepCoef<T> C, T a, T b, const OutSlot *__restrict__ slot, int flags,
              RhsSet R)
{
    const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t iy = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    int rhs;
    if (!rhs_of_slot(R, (int)blockIdx.z, rhs)) return;
    if (ix >= L.nx || iy >= L.ny) return;
    u += rhs * R.stride;
    um += rhs * R.stride;
    fre += rhs * R.stride;
    fim += rhs * R.stride;
    slot += rhs;
    const int64_t P = L.pitch;
    const int64_t i = (iy + 1) * P + L.xl + ix;
    // u_j on the 3x3 neighbourhood; first index = y offset, second = x offset
    const T umm = u[i - P - 1], um0 = u[i - P], ump = u[i - P + 1];
    const T u0m = u[i - 1], u00 = u[i], u0p = u[i + 1];
    const T upm = u[i + P - 1], up0 = u[i + P], upp = u[i + P + 1];
    // q*kappa of the four cells around the node, k<ay><ax>: cell at row y-1+ay, column x-1+ax
    const T k00 = kap[i - P - 1], k01 = kap[i - P], k10 = kap[i - 1], k11 = kap[i];
    // pair sums shared with the temporally blocked kernel (same order, same result)
    const T pm = umm + ump, p0 = u0m + u0p, pp = upm + upp;
    const T hk0 = k00 + k01, hk1 = k10 + k11;
    const Stencil2dCoef<T> SC = stencil2d_coef(C);
    const T acc = stencil2d(SC, umm, um0, ump, u0m, u00, u0p, upm, up0, upp, k00, k01, k10, k11,
                            pm, p0, pp, hk0, hk1);
    // acc + a Re F - b Im F as two FMAs (the blocked kernels round the same way)
    const T ag = vfma(a, fre[i], vfma(-b, fim[i], acc));
    const T d = dco[i];
    const T uprev = um[i];
    const T unew = vfma(d, vfma(T(-2), uprev, ag), uprev);
    um[i] = unew;
    if (flags) {
        const int64_t c = iy * L.nx + ix;
        if ((flags & 1) && slot->snap_part) slot->snap_part[2 * c] = (double)unew;
        if ((flags & 2) && slot->final_part) slot->final_part[2 * c] = (double)unew;
    }
}

// Each thread walks a column of kZChunk planes in z with a 3x3x3 register
// window of u_j (planes z-1, z, z+1) and a 2x2x2 window of cells, so a node
// costs 9 new loads of u_j and 4 of q*kappa (neighbours in x and y come from
// L1, the plane below and the node's own plane from registers).
constexpr int kZChunk = 16;

template <typename T>
__global__ void __launch_bounds__(256)
step3d_kernel(const T *__restrict__ u, T *__restrict__ um, const T *__restrict__ kap,
              const T *__restrict__ dco, const T *__restrict__ fre, const T *__restrict__ fim,
              Layout L, StepCoef<T> C, T a, T b, const OutSlot *__restrict__ slot, int flags,
              RhsSet R, int nchunks)
{
    const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t iy = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    int rhs;
    if (!rhs_of_slot(R, (int)blockIdx.z / nchunks, rhs)) return;
    const int64_t z0 = (int64_t)(blockIdx.z % nchunks) * kZChunk;
    const int64_t z1 = min((int64_t)L.nz, z0 + kZChunk);
    if (ix >= L.nx || iy >= L.ny) return;
    u += rhs * R.stride;
    um += rhs * R.stride;
    fre += rhs * R.stride;
    fim += rhs * R.stride;
    slot += rhs;
    const int64_t P = L.pitch, Q = L.plane;
    const int64_t col = (iy + 1) * P + L.xl + ix;     // (y, x) offset of the node in any plane
    // w[p][oy][ox]: u_j at stored plane (iz + p), row offset oy-1, column offset ox-1
    T w[3][3][3];
    // k[az][ay][ax]: q*kappa of the cell at stored plane (iz + az), row y-1+ay, column x-1+ax
    T k[2][2][2];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int oy = 0; oy < 3; ++oy)
#pragma unroll
            for (int ox = 0; ox < 3; ++ox)
                w[p][oy][ox] = u[(z0 + p) * Q + col + (oy - 1) * P + (ox - 1)];
#pragma unroll
    for (int ay = 0; ay < 2; ++ay)
#pragma unroll
        for (int ax = 0; ax < 2; ++ax)
            k[0][ay][ax] = kap[z0 * Q + col - (1 - ay) * P - (1 - ax)];
    for (int64_t iz = z0; iz < z1; ++iz) {
#pragma unroll
        for (int oy = 0; oy < 3; ++oy)
#pragma unroll
            for (int ox = 0; ox < 3; ++ox)
                w[2][oy][ox] = u[(iz + 2) * Q + col + (oy - 1) * P + (ox - 1)];
#pragma unroll
        for (int ay = 0; ay < 2; ++ay)
#pragma unroll
            for (int ax = 0; ax < 2; ++ax)
                k[1][ay][ax] = kap[(iz + 1) * Q + col - (1 - ay) * P - (1 - ax)];
        // sums of kappa over the cells shared by the node and its neighbour at
        // offset o - 1 (o in 0..2 per axis): -1 keeps the lower cell, +1 the upper, 0 both
        T kx[2][2][3];
#pragma unroll
        for (int az = 0; az < 2; ++az)
#pragma unroll
            for (int ay = 0; ay < 2; ++ay) {
                kx[az][ay][0] = k[az][ay][0];
                kx[az][ay][1] = k[az][ay][0] + k[az][ay][1];
                kx[az][ay][2] = k[az][ay][1];
            }
        T kxy[2][3][3];
#pragma unroll
        for (int az = 0; az < 2; ++az)
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) {
                kxy[az][0][ox] = kx[az][0][ox];
                kxy[az][1][ox] = kx[az][0][ox] + kx[az][1][ox];
                kxy[az][2][ox] = kx[az][1][ox];
            }
        T acc = T(0);
#pragma unroll
        for (int oz = 0; oz < 3; ++oz)
#pragma unroll
            for (int oy = 0; oy < 3; ++oy)
#pragma unroll
                for (int ox = 0; ox < 3; ++ox) {
                    const int s = (oz != 1) + (oy != 1) + (ox != 1);
                    const T ks = (oz == 0) ? kxy[0][oy][ox]
                               : (oz == 2) ? kxy[1][oy][ox] : kxy[0][oy][ox] + kxy[1][oy][ox];
                    const T coef = (s == 0) ? C.c0 + C.mt[0] * ks : C.mt[s] * ks - C.cs[s];
                    acc += coef * w[oz][oy][ox];
                }
        const int64_t i = (iz + 1) * Q + col;
        const T g = a * fre[i] - b * fim[i];
        const T d = dco[i];
        const T uprev = um[i];
        const T unew = d * (acc + g - T(2) * uprev) + uprev;
        um[i] = unew;
        if (flags) {
            const int64_t c = (iz * L.ny + iy) * L.nx + ix;
            if ((flags & 1) && slot->snap_part) slot->snap_part[2 * c] = (double)unew;
            if ((flags & 2) && slot->final_part) slot->final_part[2 * c] = (double)unew;
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
    }
}

template <typename T>
void launch_step(const Layout &L, const T *u, T *um, const T *kap, const T *dco,
                 const T *fre, const T *fim, const StepCoef<T> &C, T a, T b,
                 const OutSlot *slot, int flags, cudaStream_t s, const RhsSet &R)
{
    if (L.d == 2) {
        dim3 blk(32, 8);
        dim3 grd((unsigned)((L.nx + 31) / 32), (unsigned)((L.ny + 7) / 8), (unsigned)R.slots);
        step2d_kernel<T><<<grd, blk, 0, s>>>(u, um, kap, dco, fre, fim, L, C, a, b, slot, flags,
                                             R);
        ++g_launches;
    } else {
        const int nchunks = (int)((L.nz + kZChunk - 1) / kZChunk);
        dim3 blk(32, 8);
        dim3 grd((unsigned)((L.nx + 31) / 32), (unsigned)((L.ny + 7) / 8),
                 (unsigned)(nchunks * R.slots));
        step3d_kernel<T><<<grd, blk, 0, s>>>(u, um, kap, dco, fre, fim, L, C, a, b, slot, flags,
                                             R, nchunks);
        ++g_launches;
    }
}

template void launch_step<float>(const Layout &, const float *, float *, const float *,
                                 const float *, const float *, const float *,
                                 const StepCoef<float> &, float, float, const OutSlot *, int,
                                 cudaStream_t, const RhsSet &);
template void launch_step<double>(const Layout &, const double *, double *, const double *,
                                  const double *, const double *, const double *,
                                  const StepCoef<double> &, double, double, const OutSlot *,
                                  int, cudaStream_t, const RhsSet &);

// ---------------------------------------------------------------------------
// frequency-adapted backward-differences damped leapfrog (Def. of I_abd)
// ---------------------------------------------------------------------------
//
//   u_{n+1} = (2 - K - L) u_n - (I - L) u_{n-1} + g_n,
//   K = (dt^2/alpha)(Re H + omega^2) - (dt beta (1 - cos(omega dt))/alpha) B,
//   L = (beta dt/alpha) B,  B = Im H / omega,
// which regroups into
//   u_{n+1} = [2 - (dt^2/alpha)(Re H + omega^2)] u_n - u_{n-1}
//             - (beta dt/(alpha omega)) Im H (cos(omega dt) u_n - u_{n-1}) + g_n.
// The first bracket is the same h^2-scaled cell stencil as I_acd's (StepCoef,
// q*kappa per cell).  Im H: node damping omega_phys R_i (damp holds
// beta dt omega_phys R_i/(alpha omega) per node), or cell damping (damp holds
// that coefficient with R_cell per cell; the operator is the cell-mass stencil
// sum_o M_s (sum of damp over the shared cells) w_{beta+o}).  Reads u_{n-1} at
// the neighbours in the cell case, so u_{n+1} goes to a third plane.

template <typename T, int D, bool kCell>
__global__ void __launch_bounds__(256)
abd_step_kernel(const T *__restrict__ u, const T *__restrict__ um, T *__restrict__ out,
                const T *__restrict__ kap, const T *__restrict__ damp,
                const T *__restrict__ fre, const T *__restrict__ fim, Layout L, StepCoef<T> C,
                T a, T b, T cth, const OutSlot *__restrict__ slot, int flags, RhsSet R, int nz)
{
    const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t iy = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    int rhs;
    if (!rhs_of_slot(R, (int)blockIdx.z / nz, rhs)) return;
    const int64_t iz = blockIdx.z % nz;
    if (ix >= L.nx || iy >= L.ny) return;
    const int64_t off = rhs * R.stride;
    u += off;
    um += off;
    out += off;
    fre += off;
    fim += off;
    slot += rhs;
    const int64_t P = L.pitch, Q = L.plane;
    const int64_t i = L.node(ix, iy, iz);
    constexpr int NC = 1 << D;
    // the node's cells, bit t of index c: upper (1) or lower (0) cell along axis t
    // (t = 0: x, 1: y, 2: z)
    T kc[NC], dc[NC];
#pragma unroll
    for (int cidx = 0; cidx < NC; ++cidx) {
        const int ax = cidx & 1, ay = (cidx >> 1) & 1, az = (cidx >> 2) & 1;
        const int64_t ci = i - (1 - ax) - (1 - ay) * P - (D == 3 ? (1 - az) * Q : 0);
        kc[cidx] = kap[ci];
        if (kCell) dc[cidx] = damp[ci];
    }
    T accA = T(0), accB = T(0);
#pragma unroll
    for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz)
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
                const int sh = (ox != 0) + (oy != 0) + (oz != 0);
                T ks = T(0), ds = T(0);
#pragma unroll
                for (int cidx = 0; cidx < NC; ++cidx) {
                    const int ax = cidx & 1, ay = (cidx >> 1) & 1, az = (cidx >> 2) & 1;
                    const bool shared = (ox == 0 || ox == 2 * ax - 1) &&
                                        (oy == 0 || oy == 2 * ay - 1) &&
                                        (D == 2 || oz == 0 || oz == 2 * az - 1);
                    if (shared) {
                        ks += kc[cidx];
                        if (kCell) ds += dc[cidx];
                    }
                }
                const int64_t j = i + ox + oy * P + (D == 3 ? oz * Q : 0);
                const T v = u[j];
                const T coef = (sh == 0) ? C.c0 + C.mt[0] * ks : C.mt[sh] * ks - C.cs[sh];
                accA += coef * v;
                if (kCell) accB += C.mt[sh] * ds * (cth * v - um[j]);
            }
    const T prev = um[i];
    if (!kCell) accB = damp[i] * (cth * u[i] - prev);
    const T unew = accA - prev - accB + (a * fre[i] - b * fim[i]);
    out[i] = unew;
    if (flags) {
        const int64_t c = (iz * L.ny + iy) * L.nx + ix;
        if ((flags & 1) && slot->snap_part) slot->snap_part[2 * c] = (double)unew;
        if ((flags & 2) && slot->final_part) slot->final_part[2 * c] = (double)unew;
    }
}

template <typename T>
void launch_abd_step(const Layout &L, const T *u, const T *um, T *out, const T *kap,
                     const T *damp, bool cell, const T *fre, const T *fim, const StepCoef<T> &C,
                     T a, T b, T cth, const OutSlot *slot, int flags, cudaStream_t s,
                     const RhsSet &R)
{
    const int nz = (int)L.nz;
    dim3 blk(32, 8);
    dim3 grd((unsigned)((L.nx + 31) / 32), (unsigned)((L.ny + 7) / 8), (unsigned)(nz * R.slots));
#define HTD_ABD_LAUNCH(DD, CC)                                                                  \
    abd_step_kernel<T, DD, CC><<<grd, blk, 0, s>>>(u, um, out, kap, damp, fre, fim, L, C, a, b, \
                                                   cth, slot, flags, R, nz)
    if (L.d == 3) {
        if (cell) HTD_ABD_LAUNCH(3, true); else HTD_ABD_LAUNCH(3, false);
    } else {
        if (cell) HTD_ABD_LAUNCH(2, true); else HTD_ABD_LAUNCH(2, false);
    }
#undef HTD_ABD_LAUNCH
    ++g_launches;
}
template void launch_abd_step<float>(const Layout &, const float *, const float *, float *,
                                     const float *, const float *, bool, const float *,
                                     const float *, const StepCoef<float> &, float, float, float,
                                     const OutSlot *, int, cudaStream_t, const RhsSet &);
template void launch_abd_step<double>(const Layout &, const double *, const double *, double *,
                                      const double *, const double *, bool, const double *,
                                      const double *, const StepCoef<double> &, double, double,
                                      double, const OutSlot *, int, cudaStream_t, const RhsSet &);

// ---------------------------------------------------------------------------
// projection read-out: compensated sums of e^{-i theta_j} u_j
// ---------------------------------------------------------------------------

// one compensated (Kahan) addition s += x, c carrying the negated lost low part
template <typename T>
__device__ __forceinline__ void kahan_add(T &s, T &c, T x)
{
    const T y = x - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
}

// acc planes per rhs (stride apart), compact node order: [s_re, s_im, c_re, c_im]
// x N.  For the state u (padded layout) of every listed rhs:
//   s_re += wc u, s_im += ws u   (wc = cos theta, ws = -sin theta), compensated.
template <typename T>
__global__ void __launch_bounds__(256)
project_accumulate_kernel(Layout L, const T *__restrict__ u, T *__restrict__ acc, int64_t astride,
                          T wc, T ws, RhsSet R, int nz)
{
    const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t iy = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    int rhs;
    if (!rhs_of_slot(R, (int)blockIdx.z / nz, rhs)) return;
    const int64_t iz = blockIdx.z % nz;
    if (ix >= L.nx || iy >= L.ny) return;
    const int64_t c = (iz * L.ny + iy) * L.nx + ix;
    const T v = u[rhs * R.stride + L.node(ix, iy, iz)];
    T *a = acc + rhs * astride;
    T sr = a[c], si = a[L.N + c], cr = a[2 * L.N + c], ci = a[3 * L.N + c];
    kahan_add(sr, cr, wc * v);
    kahan_add(si, ci, ws * v);
    a[c] = sr;
    a[L.N + c] = si;
    a[2 * L.N + c] = cr;
    a[3 * L.N + c] = ci;
}

template <typename T>
void launch_project_accumulate(const Layout &L, const T *u, T *acc, int64_t astride, T wc, T ws,
                               const RhsSet &R, cudaStream_t s)
{
    const int nz = (int)L.nz;
    dim3 blk(32, 8);
    dim3 grd((unsigned)((L.nx + 31) / 32), (unsigned)((L.ny + 7) / 8), (unsigned)(nz * R.slots));
    project_accumulate_kernel<T><<<grd, blk, 0, s>>>(L, u, acc, astride, wc, ws, R, nz);
    ++g_launches;
}
template void launch_project_accumulate<float>(const Layout &, const float *, float *, int64_t,
                                               float, float, const RhsSet &, cudaStream_t);
template void launch_project_accumulate<double>(const Layout &, const double *, double *, int64_t,
                                                double, double, const RhsSet &, cudaStream_t);

// U = scale (s - c) into the output slot of every listed rhs (real part to
// final_part, imaginary part to snap_part), in double
template <typename T>
__global__ void __launch_bounds__(256)
project_finish_kernel(int64_t N, const T *__restrict__ acc, int64_t astride, double scale,
                      const OutSlot *__restrict__ slot, RhsSet R)
{
    int rhs;
    if (!rhs_of_slot(R, (int)blockIdx.y, rhs)) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const T *a = acc + rhs * astride;
    const OutSlot o = slot[rhs];
    const double re = scale * ((double)a[c] - (double)a[2 * N + c]);
    const double im = scale * ((double)a[N + c] - (double)a[3 * N + c]);
    if (o.final_part) o.final_part[2 * c] = re;
    if (o.snap_part) o.snap_part[2 * c] = im;
}

template <typename T>
void launch_project_finish(int64_t N, const T *acc, int64_t astride, double scale,
                           const OutSlot *slot, const RhsSet &R, cudaStream_t s)
{
    const int bs = 256;
    dim3 grd((unsigned)((N + bs - 1) / bs), (unsigned)R.slots);
    project_finish_kernel<T><<<grd, bs, 0, s>>>(N, acc, astride, scale, slot, R);
    ++g_launches;
}
template void launch_project_finish<float>(int64_t, const float *, int64_t, double,
                                           const OutSlot *, const RhsSet &, cudaStream_t);
template void launch_project_finish<double>(int64_t, const double *, int64_t, double,
                                            const OutSlot *, const RhsSet &, cudaStream_t);

// ---------------------------------------------------------------------------
// split / output slot
// ---------------------------------------------------------------------------

template <typename T>
__global__ void split_kernel(Layout L, const double2 *__restrict__ F, T *__restrict__ fre,
                             T *__restrict__ fim, int flip)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.N) return;
    const int64_t ix = c % L.nx;
    const int64_t r = c / L.nx;
    const int64_t iy = r % L.ny;
    const int64_t iz = r / L.ny;
    const int64_t i = L.node(ix, iy, iz);
    const double2 f = F[c];
    // flip: forcing -i F, whose real part is Im F and imaginary part is -Re F
    fre[i] = (T)(flip ? f.y : f.x);
    fim[i] = (T)(flip ? -f.x : f.y);
}

template <typename T>
void launch_split(const Layout &L, const double2 *F, T *fre, T *fim, int flip, cudaStream_t s)
{
    const int bs = 256;
    split_kernel<T><<<(unsigned)((L.N + bs - 1) / bs), bs, 0, s>>>(L, F, fre, fim, flip);
    ++g_launches;
}
template void launch_split<float>(const Layout &, const double2 *, float *, float *, int, cudaStream_t);
template void launch_split<double>(const Layout &, const double2 *, double *, double *, int, cudaStream_t);

// batched forms: the active rhs list act (see RhsSet) selects the slots

template <typename T>
__global__ void split_batch_kernel(Layout L, const double2 *const *__restrict__ Fp,
                                   T *__restrict__ fre, T *__restrict__ fim, int64_t stride,
                                   int flip, const int *__restrict__ act)
{
    const int k = (int)blockIdx.y;
    if (k >= act[0]) return;
    const int r = act[1 + k];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.N) return;
    const int64_t ix = c % L.nx;
    const int64_t q = c / L.nx;
    const int64_t iy = q % L.ny;
    const int64_t iz = q / L.ny;
    const int64_t i = L.node(ix, iy, iz) + r * stride;
    const double2 f = Fp[r][c];
    fre[i] = (T)(flip ? f.y : f.x);
    fim[i] = (T)(flip ? -f.x : f.y);
}

template <typename T>
void launch_split_batch(const Layout &L, const double2 *const *Fp, T *fre, T *fim, int64_t stride,
                        int flip, const int *act, int slots, cudaStream_t s)
{
    const int bs = 256;
    dim3 grd((unsigned)((L.N + bs - 1) / bs), (unsigned)slots);
    split_batch_kernel<T><<<grd, bs, 0, s>>>(L, Fp, fre, fim, stride, flip, act);
    ++g_launches;
}
template void launch_split_batch<float>(const Layout &, const double2 *const *, float *, float *,
                                        int64_t, int, const int *, int, cudaStream_t);
template void launch_split_batch<double>(const Layout &, const double2 *const *, double *, double *,
                                         int64_t, int, const int *, int, cudaStream_t);

struct ActList {
    int n;
    int idx[kMaxRhs];
};

__global__ void set_act_kernel(int *act, ActList a)
{
    const int t = threadIdx.x;
    if (t == 0) act[0] = a.n;
    if (t < a.n) act[1 + t] = a.idx[t];
}

void launch_set_act(int *act, int n, const int *idx, cudaStream_t s)
{
    ActList a;
    a.n = n;
    for (int k = 0; k < n && k < kMaxRhs; ++k) a.idx[k] = idx[k];
    for (int k = n; k < kMaxRhs; ++k) a.idx[k] = 0;
    set_act_kernel<<<1, kMaxRhs, 0, s>>>(act, a);
    ++g_launches;
}

// output slots of the listed rhs r: the final state of run `run` goes to the
// real (run 0) or imaginary (run 1) part of Up[r]; with one run (Table 1) the
// snapshot goes to the imaginary part
__global__ void set_slots_kernel(OutSlot *slot, double2 *const *Up, int run, int runs,
                                 const int *act)
{
    const int k = threadIdx.x;
    if (k >= act[0]) return;
    const int r = act[1 + k];
    double *base = reinterpret_cast<double *>(Up[r]);
    slot[r].final_part = base + run;
    slot[r].snap_part = (runs == 1) ? base + 1 : nullptr;
}

void launch_set_slots(OutSlot *slot, double2 *const *Up, int run, int runs, const int *act,
                      int slots, cudaStream_t s)
{
    set_slots_kernel<<<1, slots, 0, s>>>(slot, Up, run, runs, act);
    ++g_launches;
}

__global__ void set_slot_kernel(OutSlot *slot, double *final_part, double *snap_part)
{
    slot->final_part = final_part;
    slot->snap_part = snap_part;
}

void launch_set_slot(OutSlot *slot, double *final_part, double *snap_part, cudaStream_t s)
{
    set_slot_kernel<<<1, 1, 0, s>>>(slot, final_part, snap_part);
    ++g_launches;
}

// ---------------------------------------------------------------------------
// true operator, complex128
// ---------------------------------------------------------------------------

struct HCoef {
    double S2[4];   // 2^{d-s} S_s
    double M[4];
};

// Linear index of the offset (oz, oy, ox) in {-1,0,1}^3: (oz+1) 9 + (oy+1) 3 + (ox+1);
// the centre is 13.  H is symmetric, so only the centre and the offsets with a
// larger index ("positive": first non-zero of (oz, oy, ox) is +1) are stored:
// plane lin - 13.  The coefficient of a negative offset o at node beta is the
// stored coefficient of -o at the node beta + o.
__host__ __device__ constexpr int hlin(int oz, int oy, int ox)
{
    return (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1);
}

// plane p (0 = centre, 1..13 positive offsets; 2-D: oz = 0, planes 0..4) of
// node (ix, iy, iz): 2^{d-s} S_s - M_s * (sum of kappa over the cells that
// contain the node and its neighbour), not yet scaled by 1/h^2; 0 where the
// neighbour is outside the grid
__global__ void __launch_bounds__(256)
assemble_H_kernel(Layout L, const double *__restrict__ kap64, HCoef C, double *__restrict__ coefP,
                  int nplanes)
{
    const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t iy = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    const int64_t iz = blockIdx.z;
    if (ix >= L.nx || iy >= L.ny) return;
    const int64_t c = (iz * L.ny + iy) * L.nx + ix;
    const int64_t i = L.node(ix, iy, iz);    // position in the padded cell array
    const int64_t P = L.pitch, Q = L.plane;
    for (int p = 0; p < nplanes; ++p) {
        const int lin = p + 13;
        const int oz = lin / 9 - 1, oy = (lin / 3) % 3 - 1, ox = lin % 3 - 1;
        const int64_t jz = iz + oz, jy = iy + oy, jx = ix + ox;
        double w = 0.0;
        if (jz >= 0 && jz < L.nz && jy >= 0 && jy < L.ny && jx >= 0 && jx < L.nx) {
            const int s = (oz != 0) + (oy != 0) + (ox != 0);
            // cells shared by the node and its neighbour: lower (offset -1), upper
            // (+1) or both (0) per axis
            double ks = 0.0;
            for (int az = (L.d == 3 ? 0 : 1); az < 2; ++az) {
                if (L.d == 3 && ((oz < 0 && az == 1) || (oz > 0 && az == 0))) continue;
                for (int ay = 0; ay < 2; ++ay) {
                    if ((oy < 0 && ay == 1) || (oy > 0 && ay == 0)) continue;
                    for (int ax = 0; ax < 2; ++ax) {
                        if ((ox < 0 && ax == 1) || (ox > 0 && ax == 0)) continue;
                        ks += kap64[i - (L.d == 3 ? (1 - az) * Q : 0) - (1 - ay) * P - (1 - ax)];
                    }
                }
            }
            w = C.S2[s] - C.M[s] * ks;
        }
        coefP[p * L.N + c] = w;
    }
}

void launch_assemble_H(const Layout &L, const double *kap64, const double S2[4], const double M[4],
                       double *coefP, cudaStream_t s)
{
    HCoef C;
    for (int k = 0; k < 4; ++k) { C.S2[k] = S2[k]; C.M[k] = M[k]; }
    dim3 blk(32, 8);
    dim3 grd((unsigned)((L.nx + 31) / 32), (unsigned)((L.ny + 7) / 8), (unsigned)L.nz);
    assemble_H_kernel<<<grd, blk, 0, s>>>(L, kap64, C, coefP, h_planes(L.d));
    ++g_launches;
}

// Y = H X (or F - H X) from the assembled coefficients: per node 3^D
// coefficient x neighbour products for the real and the imaginary part, one
// FP64 FMA each; neighbours outside the grid are the zero Dirichlet ghosts
template <int D, bool kImH>
__global__ void __launch_bounds__(256)
apply_H_asm_kernel(int64_t nx, int64_t ny, int64_t nz, const double *__restrict__ coefP,
                   const double *__restrict__ coefI, const double *__restrict__ imH, double ih2,
                   const double2 *__restrict__ X, const double2 *__restrict__ F,
                   double2 *__restrict__ Y)
{
    const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t iy = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    const int64_t iz = blockIdx.z;
    if (ix >= nx || iy >= ny) return;
    const int64_t N = nx * ny * nz;
    const int64_t c = (iz * ny + iy) * nx + ix;
    double re = 0.0, im = 0.0, qr = 0.0, qi = 0.0;
#pragma unroll
    for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz)
#pragma unroll
        for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
                const bool in = iz + oz >= 0 && iz + oz < nz && iy + oy >= 0 && iy + oy < ny &&
                                ix + ox >= 0 && ix + ox < nx;
                if (!in) continue;
                const int64_t cn = c + ((int64_t)oz * ny + oy) * nx + ox;
                const int lin = hlin(oz, oy, ox);
                const int64_t ci = (lin >= 13) ? (lin - 13) * N + c : (13 - lin) * N + cn;
                const double w = coefP[ci];
                const double2 x = X[cn];
                re = fma(w, x.x, re);
                im = fma(w, x.y, im);
                if (kImH) {                       // non-diagonal Im H (cell damping)
                    const double wi = coefI[ci];
                    qr = fma(wi, x.x, qr);
                    qi = fma(wi, x.y, qi);
                }
            }
    const double2 xc = X[c];
    const double damp = imH[c];
    double2 y;
    // H x = (Re H x_r - Im H x_i) + i (Re H x_i + Im H x_r)
    y.x = ih2 * re - damp * xc.y - qi;
    y.y = ih2 * im + damp * xc.x + qr;
    if (F) {
        const double2 f = F[c];
        y.x = f.x - y.x;
        y.y = f.y - y.y;
    }
    Y[c] = y;
}

void launch_apply_H(const Layout &L, const double *coefP, const double *imH, double ih2,
                    const double2 *X, const double2 *F, double2 *Y, cudaStream_t s,
                    const double *coefI)
{
    dim3 blk(32, 8);
    dim3 grd((unsigned)((L.nx + 31) / 32), (unsigned)((L.ny + 7) / 8), (unsigned)L.nz);
#define HTD_AH(DD, II) \
    apply_H_asm_kernel<DD, II><<<grd, blk, 0, s>>>(L.nx, L.ny, L.nz, coefP, coefI, imH, ih2, X, F, Y)
    if (L.d == 3) {
        if (coefI) HTD_AH(3, true); else HTD_AH(3, false);
    } else {
        if (coefI) HTD_AH(2, true); else HTD_AH(2, false);
    }
#undef HTD_AH
    ++g_launches;
}

// ---------------------------------------------------------------------------
// Krylov vector operations (complex128)
// ---------------------------------------------------------------------------

constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum of (re, im); result valid in thread 0
__device__ __forceinline__ double2 block_sum(double re, double im)
{
    __shared__ double sre[kRedThreads / 32], sim[kRedThreads / 32];
    re = warp_sum(re);
    im = warp_sum(im);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sre[warp] = re; sim[warp] = im; }
    __syncthreads();
    double2 out = make_double2(0.0, 0.0);
    if (warp == 0) {
        re = lane < kRedThreads / 32 ? sre[lane] : 0.0;
        im = lane < kRedThreads / 32 ? sim[lane] : 0.0;
        re = warp_sum(re);
        im = warp_sum(im);
        out = make_double2(re, im);
    }
    return out;
}

// One pass over the data for a group of up to kDotGroup basis vectors: each
// thread reads w[i] once and accumulates conj(V_k[i]) w[i] for the group, two
// elements per loop trip (more loads in flight).  Every complex product costs
// four FP64 FMAs on GB300's narrow FP64 pipe, so the kernel is FP64-bound; the
// block's 2 x kDotGroup sums are reduced together at the end.
constexpr int kDotGroup = 8;

// (re, im) += conj(a) b as four FP64 FMAs
__device__ __forceinline__ void cmac_conj(double &re, double &im, double2 a, double2 b)
{
    re = fma(a.x, b.x, re);
    re = fma(a.y, b.y, re);
    im = fma(a.x, b.y, im);
    im = fma(-a.y, b.x, im);
}

__global__ void __launch_bounds__(kRedThreads)
dots_kernel(const double2 *__restrict__ V, int64_t ldv, int kcount, const double2 *__restrict__ w,
            int64_t N, double2 *__restrict__ partial, int nb)
{
    const int k0 = blockIdx.y * kDotGroup;
    const int kn = min(kDotGroup, kcount - k0);
    double re[kDotGroup], im[kDotGroup];
#pragma unroll
    for (int q = 0; q < kDotGroup; ++q) { re[q] = 0.0; im[q] = 0.0; }
    const int64_t stride = (int64_t)nb * kRedThreads;
    int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x;
    for (; i + stride < N; i += 2 * stride) {
        const double2 b0 = w[i], b1 = w[i + stride];
#pragma unroll
        for (int q = 0; q < kDotGroup; ++q) {
            if (q < kn) {
                const double2 *vq = V + (int64_t)(k0 + q) * ldv;
                const double2 a0 = vq[i], a1 = vq[i + stride];
                cmac_conj(re[q], im[q], a0, b0);
                cmac_conj(re[q], im[q], a1, b1);
            }
        }
    }
    if (i < N) {
        const double2 b = w[i];
#pragma unroll
        for (int q = 0; q < kDotGroup; ++q)
            if (q < kn) cmac_conj(re[q], im[q], V[(int64_t)(k0 + q) * ldv + i], b);
    }
    // block reduction of all 2 x kDotGroup sums: within warps, then across warps
    __shared__ double red[kRedThreads / 32][2 * kDotGroup];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kDotGroup; ++q) {
        const double r = warp_sum(re[q]), m = warp_sum(im[q]);
        if (lane == 0) {
            red[warp][2 * q] = r;
            red[warp][2 * q + 1] = m;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * kDotGroup && (int)threadIdx.x / 2 < kn) {
        double t = 0.0;
#pragma unroll
        for (int wv = 0; wv < kRedThreads / 32; ++wv) t += red[wv][threadIdx.x];
        double *out = reinterpret_cast<double *>(partial + (int64_t)(k0 + threadIdx.x / 2) * nb +
                                                 blockIdx.x);
        out[threadIdx.x & 1] = t;
    }
}

int dots_blocks(int64_t N)
{
    // 4 blocks per SM of the current device, looked up once per device
    static int sm_count[64] = {0};
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        dev = -1;
    }
    if (dev >= 0 && sm_count[dev] > 0) {
        nsm = sm_count[dev];
    } else if (dev >= 0 &&
               cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
               nsm > 0) {
        sm_count[dev] = nsm;
    } else {
        (void)cudaGetLastError();
        nsm = 1;
    }
    const int64_t cap = std::min<int64_t>(4 * (int64_t)nsm, kMaxDotBlocks);
    int64_t nb = (N + 8 * kRedThreads - 1) / (8 * kRedThreads);
    if (nb > cap) nb = cap;
    if (nb < 1) nb = 1;
    return (int)nb;
}

void launch_dots(const double2 *V, int64_t ldv, int kcount, const double2 *w, int64_t N,
                 double2 *partial, int nb, cudaStream_t s)
{
    dim3 grd((unsigned)nb, (unsigned)((kcount + kDotGroup - 1) / kDotGroup));
    dots_kernel<<<grd, kRedThreads, 0, s>>>(V, ldv, kcount, w, N, partial, nb);
    ++g_launches;
}

__global__ void __launch_bounds__(kRedThreads)
reduce_kernel(const double2 *__restrict__ partial, int nb, double2 *__restrict__ out)
{
    const int k = blockIdx.x;
    double re = 0.0, im = 0.0;
    for (int b = threadIdx.x; b < nb; b += kRedThreads) {
        const double2 p = partial[(int64_t)k * nb + b];
        re += p.x;
        im += p.y;
    }
    const double2 t = block_sum(re, im);
    if (threadIdx.x == 0) out[k] = t;
}

void launch_reduce(const double2 *partial, int nb, int kcount, double2 *out, cudaStream_t s)
{
    reduce_kernel<<<kcount, kRedThreads, 0, s>>>(partial, nb, out);
    ++g_launches;
}

// w -= sum_k h_k V_k and U += sum_k y_k Z_k: two elements per thread (256
// apart, so that loads stay coalesced) for two independent FP64 chains, four
// FMAs per complex product
constexpr int kCombThreads = 256;

template <bool kAdd>
__global__ void __launch_bounds__(kCombThreads)
combination_kernel(const double2 *__restrict__ V, int64_t ldv, int kcount,
                   const double2 *__restrict__ h, double2 *__restrict__ w, int64_t N)
{
    __shared__ double2 sh[72];
    for (int k = threadIdx.x; k < kcount; k += blockDim.x) sh[k] = h[k];
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * (2 * kCombThreads) + threadIdx.x;
    const int64_t i1 = i0 + kCombThreads;
    const bool has1 = i1 < N;
    if (i0 >= N) return;
    double2 acc0 = w[i0];
    double2 acc1 = has1 ? w[i1] : make_double2(0.0, 0.0);
#pragma unroll 4
    for (int k = 0; k < kcount; ++k) {
        const double2 *vk = V + (int64_t)k * ldv;
        const double2 c = sh[k];
        const double cx = kAdd ? c.x : -c.x, cy = kAdd ? c.y : -c.y;
        const double2 v0 = vk[i0];
        const double2 v1 = has1 ? vk[i1] : make_double2(0.0, 0.0);
        acc0.x = fma(cx, v0.x, acc0.x);
        acc0.x = fma(-cy, v0.y, acc0.x);
        acc0.y = fma(cx, v0.y, acc0.y);
        acc0.y = fma(cy, v0.x, acc0.y);
        acc1.x = fma(cx, v1.x, acc1.x);
        acc1.x = fma(-cy, v1.y, acc1.x);
        acc1.y = fma(cx, v1.y, acc1.y);
        acc1.y = fma(cy, v1.x, acc1.y);
    }
    w[i0] = acc0;
    if (has1) w[i1] = acc1;
}

void launch_sub_combination(const double2 *V, int64_t ldv, int kcount, const double2 *h,
                            double2 *w, int64_t N, cudaStream_t s)
{
    const unsigned nblk = (unsigned)((N + 2 * kCombThreads - 1) / (2 * kCombThreads));
    combination_kernel<false><<<nblk, kCombThreads, 0, s>>>(V, ldv, kcount, h, w, N);
    ++g_launches;
}

void launch_add_combination(const double2 *Z, int64_t ldz, int kcount, const double2 *y,
                            double2 *U, int64_t N, cudaStream_t s)
{
    const unsigned nblk = (unsigned)((N + 2 * kCombThreads - 1) / (2 * kCombThreads));
    combination_kernel<true><<<nblk, kCombThreads, 0, s>>>(Z, ldz, kcount, y, U, N);
    ++g_launches;
}

__global__ void scale_kernel(const double2 *__restrict__ w, double scale, double2 *__restrict__ v,
                             int64_t N)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 a = w[i];
    v[i] = make_double2(a.x * scale, a.y * scale);
}

__global__ void scale_inplace_kernel(double2 *__restrict__ v, double scale, int64_t N)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 a = v[i];
    v[i] = make_double2(a.x * scale, a.y * scale);
}

void launch_scale(const double2 *w, double scale, double2 *v, int64_t N, cudaStream_t s)
{
    const int bs = 256;
    if (w == v) {
        scale_inplace_kernel<<<(unsigned)((N + bs - 1) / bs), bs, 0, s>>>(v, scale, N);
        ++g_launches;
        return;
    }
    scale_kernel<<<(unsigned)((N + bs - 1) / bs), bs, 0, s>>>(w, scale, v, N);
    ++g_launches;
}

}  // namespace htd

namespace htd {

// ---------------------------------------------------------------------------
// receiver misfit and gradient (adjoint state)
// ---------------------------------------------------------------------------

__global__ void gather_residual_kernel(const double2 *__restrict__ U, const double2 *__restrict__ d,
                                       const int64_t *__restrict__ rec, int nrec,
                                       double2 *__restrict__ res)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrec) return;
    const double2 u = U[rec[k]], dd = d[k];
    res[k] = make_double2(u.x - dd.x, u.y - dd.y);
}

__global__ void scatter_conj_kernel(const double2 *__restrict__ res, const int64_t *__restrict__ rec,
                                    int nrec, double2 *__restrict__ r)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrec) return;
    double *p = reinterpret_cast<double *>(r + rec[k]);
    atomicAdd(p, res[k].x);          // receivers may repeat: accumulate conj(res)
    atomicAdd(p + 1, -res[k].y);
}

void launch_receiver_residual(const double2 *U, const double2 *d, const int64_t *rec, int nrec,
                              double2 *res, double2 *r, cudaStream_t s)
{
    if (nrec <= 0) return;
    const int bs = 256;
    gather_residual_kernel<<<(nrec + bs - 1) / bs, bs, 0, s>>>(U, d, rec, nrec, res);
    ++g_launches;
    scatter_conj_kernel<<<(nrec + bs - 1) / bs, bs, 0, s>>>(res, rec, nrec, r);
    ++g_launches;
}

// ---- gradient through the recurrence (htd_grad_td) --------------------------

// res[k] = U[rec[k]] - d[k]; adjoint forcing planes (padded, pre-zeroed):
// are[node(rec)] += Re res, aim[node(rec)] += Im res (receivers may repeat)
template <typename T>
__global__ void residual_planes_kernel(Layout L, const double2 *__restrict__ U,
                                       const double2 *__restrict__ d,
                                       const int64_t *__restrict__ rec, int nrec,
                                       double2 *__restrict__ res, T *__restrict__ are,
                                       T *__restrict__ aim)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrec) return;
    const int64_t c = rec[k];
    const double2 u = U[c], dd = d[k];
    const double2 r = make_double2(u.x - dd.x, u.y - dd.y);
    res[k] = r;
    const int64_t ix = c % L.nx, q = c / L.nx, iy = q % L.ny, iz = q / L.ny;
    const int64_t i = L.node(ix, iy, iz);
    atomicAdd(are + i, (T)r.x);
    atomicAdd(aim + i, (T)r.y);
}

template <typename T>
void launch_residual_planes(const Layout &L, const double2 *U, const double2 *d,
                            const int64_t *rec, int nrec, double2 *res, T *are, T *aim,
                            cudaStream_t s)
{
    if (nrec <= 0) return;
    const int bs = 256;
    residual_planes_kernel<T><<<(nrec + bs - 1) / bs, bs, 0, s>>>(L, U, d, rec, nrec, res, are,
                                                                   aim);
    ++g_launches;
}
template void launch_residual_planes<float>(const Layout &, const double2 *, const double2 *,
                                            const int64_t *, int, double2 *, float *, float *,
                                            cudaStream_t);
template void launch_residual_planes<double>(const Layout &, const double2 *, const double2 *,
                                             const int64_t *, int, double2 *, double *, double *,
                                             cudaStream_t);

template <typename T>
struct TdGradCoef {
    T M[4];
    double cm;      // -(dt^2/alpha) omega_phys^2
    double cR;      // beta dt omega_phys / (2 alpha omega)
};

// One term of the gradient sum, for the multiplier lam = lam_k and the states
// u_k, u_{k-1}, u_{k-2} (all padded; the ghost ring is zero):
//   gm[cell] += cm sum_{b,g corners} lam_b M_{|b-g|} u_{k-1,g}
//   gR[node] += cR lam (u_k - u_{k-2})
// One thread per cell (compact (n+1)^d order); the thread of cell a >= 0 also
// does node a.  Products in the recurrence precision, sums in double.
template <typename T, int D>
__global__ void __launch_bounds__(256)
grad_td_kernel(Layout L, TdGradCoef<T> G, const T *__restrict__ lam, const T *__restrict__ uk,
               const T *__restrict__ uk1, const T *__restrict__ uk2, double *__restrict__ gm,
               double *__restrict__ gR)
{
    const int64_t cx_n = L.nx + 1, cy_n = L.ny + 1, cz_n = (D == 3) ? L.nz + 1 : 1;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cx_n * cy_n * cz_n) return;
    const int64_t ax = c % cx_n - 1;
    const int64_t rr = c / cx_n;
    const int64_t ay = rr % cy_n - 1;
    const int64_t az = (D == 3) ? rr / cy_n - 1 : 0;
    constexpr int nc = (D == 3) ? 8 : 4;
    if (gm) {
        T l8[nc], u8[nc];
#pragma unroll
        for (int b = 0; b < nc; ++b) {
            const int64_t i = L.node(ax + (b & 1), ay + ((b >> 1) & 1), az + ((b >> 2) & 1));
            l8[b] = lam[i];
            u8[b] = uk1[i];
        }
        T acc = T(0);
#pragma unroll
        for (int b = 0; b < nc; ++b) {
            T row = T(0);
#pragma unroll
            for (int g = 0; g < nc; ++g) row += G.M[__popc(b ^ g)] * u8[g];
            acc += l8[b] * row;
        }
        gm[c] += G.cm * (double)acc;
    }
    if (gR && ax >= 0 && ay >= 0 && (D == 2 || az >= 0) && ax < L.nx && ay < L.ny &&
        (D == 2 || az < L.nz)) {
        const int64_t i = L.node(ax, ay, az);
        const int64_t n = (az * L.ny + ay) * L.nx + ax;
        gR[n] += G.cR * (double)(lam[i] * (uk[i] - uk2[i]));
    }
}

template <typename T>
void launch_grad_td(const Layout &L, const double M[4], double cm, double cR, const T *lam,
                    const T *uk, const T *uk1, const T *uk2, double *gm, double *gR,
                    cudaStream_t s)
{
    TdGradCoef<T> G;
    for (int k = 0; k < 4; ++k) G.M[k] = (T)M[k];
    G.cm = cm;
    G.cR = cR;
    const int64_t ncell = (L.nx + 1) * (L.ny + 1) * ((L.d == 3) ? L.nz + 1 : 1);
    const int bs = 256;
    if (L.d == 3)
        grad_td_kernel<T, 3><<<(unsigned)((ncell + bs - 1) / bs), bs, 0, s>>>(L, G, lam, uk, uk1,
                                                                             uk2, gm, gR);
    else
        grad_td_kernel<T, 2><<<(unsigned)((ncell + bs - 1) / bs), bs, 0, s>>>(L, G, lam, uk, uk1,
                                                                             uk2, gm, gR);
    ++g_launches;
}
template void launch_grad_td<float>(const Layout &, const double[4], double, double, const float *,
                                    const float *, const float *, const float *, double *,
                                    double *, cudaStream_t);
template void launch_grad_td<double>(const Layout &, const double[4], double, double,
                                     const double *, const double *, const double *,
                                     const double *, double *, double *, cudaStream_t);

struct GradCoef {
    double M[4];
    double w2;      // omega_phys^2
    double w;       // omega_phys
};

// per cell alpha: gm[alpha] += omega^2 Re sum_{beta,gamma in cell} mu_beta M_{|beta-gamma|} U_gamma
// (cells in the compact (n+1)^d order of the speed input; ghost corners are zero)
__global__ void __launch_bounds__(256)
grad_cells_kernel(Layout L, GradCoef G, const double2 *__restrict__ mu,
                  const double2 *__restrict__ U, double *__restrict__ gm)
{
    const int64_t cx_n = L.nx + 1, cy_n = L.ny + 1, cz_n = (L.d == 3) ? L.nz + 1 : 1;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cx_n * cy_n * cz_n) return;
    const int64_t ax = c % cx_n - 1;
    const int64_t rr = c / cx_n;
    const int64_t ay = rr % cy_n - 1;
    const int64_t az = (L.d == 3) ? rr / cy_n - 1 : 0;
    const int nc = (L.d == 3) ? 8 : 4;
    double2 m8[8], u8[8];
    for (int b = 0; b < nc; ++b) {
        const int64_t x = ax + (b & 1), y = ay + ((b >> 1) & 1), z = az + ((b >> 2) & 1);
        const bool in = x >= 0 && x < L.nx && y >= 0 && y < L.ny && z >= 0 && z < L.nz;
        const int64_t i = (z * L.ny + y) * L.nx + x;
        m8[b] = in ? mu[i] : make_double2(0.0, 0.0);
        u8[b] = in ? U[i] : make_double2(0.0, 0.0);
    }
    double acc = 0.0;
    for (int b = 0; b < nc; ++b)
        for (int g = 0; g < nc; ++g) {
            const double wgt = G.M[__popc(b ^ g)];
            acc += wgt * (m8[b].x * u8[g].x - m8[b].y * u8[g].y);   // Re(mu_b U_g)
        }
    gm[c] += G.w2 * acc;
}

// per node: gR[i] += omega Im(mu_i U_i)
__global__ void grad_nodes_kernel(int64_t N, double w, const double2 *__restrict__ mu,
                                  const double2 *__restrict__ U, double *__restrict__ gR)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double2 a = mu[i], b = U[i];
    gR[i] += w * (a.x * b.y + a.y * b.x);
}

void launch_gradients(const Layout &L, const double M[4], double omega_phys, const double2 *mu,
                      const double2 *U, double *gm, double *gR, cudaStream_t s)
{
    GradCoef G;
    for (int k = 0; k < 4; ++k) G.M[k] = M[k];
    G.w2 = omega_phys * omega_phys;
    G.w = omega_phys;
    const int bs = 256;
    if (gm) {
        const int64_t ncell = (L.nx + 1) * (L.ny + 1) * ((L.d == 3) ? L.nz + 1 : 1);
        grad_cells_kernel<<<(unsigned)((ncell + bs - 1) / bs), bs, 0, s>>>(L, G, mu, U, gm);
        ++g_launches;
    }
    if (gR) {
        grad_nodes_kernel<<<(unsigned)((L.N + bs - 1) / bs), bs, 0, s>>>(L.N, omega_phys, mu, U, gR);
        ++g_launches;
    }
}

}  // namespace htd
