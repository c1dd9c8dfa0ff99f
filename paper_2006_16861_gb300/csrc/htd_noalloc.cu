// Allocation-free residual norm (htd_residual_norm_noalloc, include/htd.h).
//
// For callers that must not allocate device memory when they call us: code
// running under a CUDA stream capture (cudaMalloc is not permitted during a
// global-mode capture) and applications that own all device memory through
// their own pool and forbid libraries to cudaMalloc/cudaFree in their solve
// loop.  The ordinary htd_residual_norm keeps its residual vector and partial
// sums in the handle's cudaMalloc'd workspace; this variant keeps them in the
// fixed static buffer below, so the call itself allocates nothing.  The paper
// has no counterpart; the arithmetic is that of htd_residual_norm (the same
// operator and reduction kernels).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "htd.h"
#include "htd_internal.h"

namespace {

constexpr int kMaxPartials = 1216;    // upper bound of htd::dots_blocks()
constexpr int kMaxDevices = 64;

// Layout of the buffer (complex128 units):
//   [0, HTD_NOALLOC_MAX_NODES)           residual r = F - H U
//   next 2 * kMaxPartials                block partial sums of ||r||^2, ||F||^2
//   next 2                               the two reduced sums
constexpr size_t kScratchElems = (size_t)HTD_NOALLOC_MAX_NODES + 2 * kMaxPartials + 2;

// Every GPU that loads the library holds this array (about 4.04 MiB) until
// the process exits.  Host code must not pass the symbol itself to a kernel:
// on the host it names a host-side stand-in, not device memory.
static __device__ __align__(256) double2 g_noalloc_scratch[kScratchElems];

std::mutex g_setup_mu;
double2 *g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of the buffer on the current device, looked up once per
// device (the lookup may load the module, so it must not run under capture).
htd_status scratch_address(int dev, double2 **out)
{
    if (dev < 0 || dev >= kMaxDevices) return HTD_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            (void)cudaGetLastError();
            return HTD_ERR_CUDA;
        }
        g_scratch_dev[dev] = static_cast<double2 *>(ptr);
    }
    *out = g_scratch_dev[dev];
    return HTD_OK;
}

}  // namespace

extern "C" htd_status htd_residual_norm_noalloc(htd_handle h, const void *F_dev, const void *U_dev,
                                                double *rel, void *stream)
{
    if (!h || !F_dev || !U_dev || !rel) return HTD_ERR_ARG;
    htd::OperatorView op;
    htd::operator_view(h, &op);
    const int64_t N = op.L64.N;
    if (N > HTD_NOALLOC_MAX_NODES) return HTD_ERR_SIZE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return HTD_ERR_CUDA;
    }
    if (dev != op.device) return HTD_ERR_ARG;
    double2 *base = nullptr;
    htd_status st = scratch_address(dev, &base);
    if (st != HTD_OK) return st;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double2 *r = base;
    double2 *partial = base + HTD_NOALLOC_MAX_NODES;
    double2 *sums = partial + 2 * kMaxPartials;
    const int nb = htd::dots_blocks(N);
    if (nb > kMaxPartials) return HTD_ERR_SIZE;

    // every element read below is written first by this call: r by apply_H,
    // the partials by the dot kernels, the sums by the reductions
    htd::launch_apply_H(op.L64, op.coefP, op.imH, op.ih2,
                        static_cast<const double2 *>(U_dev), static_cast<const double2 *>(F_dev),
                        r, s, op.coefI);
    htd::launch_dots(r, N, 1, r, N, partial, nb, s);
    htd::launch_reduce(partial, nb, 1, sums, s);
    htd::launch_dots(static_cast<const double2 *>(F_dev), N, 1,
                     static_cast<const double2 *>(F_dev), N, partial + kMaxPartials, nb, s);
    htd::launch_reduce(partial + kMaxPartials, nb, 1, sums + 1, s);
    double2 host[2];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, sums, sizeof(host), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return HTD_ERR_CUDA;
    }
    const double rr = host[0].x, ff = host[1].x;
    if (!std::isfinite(rr) || !std::isfinite(ff)) return HTD_ERR_NONFINITE;
    *rel = (ff > 0.0) ? std::sqrt(rr > 0.0 ? rr : 0.0) / std::sqrt(ff) : 0.0;
    return HTD_OK;
}
