// Internal declarations shared by the libhtd translation units.
// Not part of the public ABI (include/htd.h is).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

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

// Output targets of a preconditioner run, read by the step kernels from device
// memory so that a captured graph can be replayed for any output vector.
struct OutSlot {
    double *final_part;   // &U[0].re or &U[0].im (stride 2 doubles), or null
    double *snap_part;    // &U[0].im (stride 2), or null
};

// ---- kernel launchers (htd_kernels.cu) --------------------------------------

// Number of kernels enqueued by this library (host counter, not thread-safe
// across handles used concurrently; used for statistics only).
extern long long g_launches;

template <typename T>
void launch_step(const Layout &L, const T *u, T *um, const T *kap, const T *dco,
                 const T *fre, const T *fim, const StepCoef<T> &C, T a, T b,
                 const OutSlot *slot, int flags, cudaStream_t s);

template <typename T>
void launch_split(const Layout &L, const double2 *F, T *fre, T *fim, int flip, cudaStream_t s);

void launch_set_slot(OutSlot *slot, double *final_part, double *snap_part, cudaStream_t s);

// Y = H X (F == null) or Y = F - H X, complex128 compact vectors.
void launch_apply_H(const Layout &L, const double *kap64, const double *imH,
                    const double S2[4], const double M[4], double ih2,
                    const double2 *X, const double2 *F, double2 *Y, cudaStream_t s);

// partial[k * nb + b] = sum over block b of conj(V_k) w, k < kcount
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
// v = w * scale
void launch_scale(const double2 *w, double scale, double2 *v, int64_t N, cudaStream_t s);

// Read-only view of a handle's FP64 operator data (defined in htd_capi.cu).
struct OperatorView {
    Layout L64;             // layout of kap64 (compact N = L64.N)
    const double *kap64;    // (h k)^2 per cell
    const double *imH;      // omega_phys R per node
    double S2[4], M[4], ih2;
    int device;
};
void operator_view(const htd_ctx *c, OperatorView *out);

}  // namespace htd
