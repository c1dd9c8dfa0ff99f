// Allocation-free residual norm (htd_residual_norm_noalloc, include/htd.h).
//
// For callers that cannot let a library allocate device memory when they call
// it: applications whose device memory is handed out by their own pool (a
// framework's caching allocator that has reserved most of the GPU, where a
// library's cudaMalloc would fail or fragment it) and solve loops that cannot
// afford the device-wide synchronisation cudaMalloc/cudaFree may imply while
// other streams run.  The ordinary htd_residual_norm keeps its residual vector
// and partial sums in the handle's cudaMalloc'd workspace; this variant keeps
// them in the fixed static buffer below, so the call itself allocates nothing.
// It synchronises the stream it is given (it returns a host value), so it is
// not for use inside a stream capture.  The paper has no counterpart; the
// arithmetic is that of htd_residual_norm (the same operator and reduction
// kernels).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "htd.h"
#include "htd_internal.h"

namespace {

constexpr int kMaxPartials = htd::kMaxDotBlocks;   // upper bound of htd::dots_blocks()
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

// After a CUDA error the context may have been reset or lost; the next call on
// this device looks the address up again instead of trusting the cached one.
void forget_address(int dev)
{
    if (dev < 0 || dev >= kMaxDevices) return;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    g_scratch_dev[dev] = nullptr;
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
    // an error left pending by earlier work is reported, not cleared, and
    // nothing is launched: it is not this call's to swallow
    if (cudaPeekAtLastError() != cudaSuccess) return HTD_ERR_CUDA;
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
    auto failed = [&](cudaError_t e) {
        if (e == cudaSuccess) return false;
        (void)cudaGetLastError();
        forget_address(dev);
        return true;
    };

    // every element read below is written first by this call: r by apply_H,
    // the partials by the dot kernels, the sums by the reductions; each
    // launch is checked as soon as it is made
    htd::launch_apply_H(op.L64, op.coefP, op.imH, op.ih2,
                        static_cast<const double2 *>(U_dev), static_cast<const double2 *>(F_dev),
                        r, s, op.coefI);
    if (failed(cudaGetLastError())) return HTD_ERR_CUDA;
    htd::launch_dots(r, N, 1, r, N, partial, nb, s);
    if (failed(cudaGetLastError())) return HTD_ERR_CUDA;
    htd::launch_reduce(partial, nb, 1, sums, s);
    if (failed(cudaGetLastError())) return HTD_ERR_CUDA;
    htd::launch_dots(static_cast<const double2 *>(F_dev), N, 1,
                     static_cast<const double2 *>(F_dev), N, partial + kMaxPartials, nb, s);
    if (failed(cudaGetLastError())) return HTD_ERR_CUDA;
    htd::launch_reduce(partial + kMaxPartials, nb, 1, sums + 1, s);
    if (failed(cudaGetLastError())) return HTD_ERR_CUDA;
    double2 host[2];
    if (failed(cudaMemcpyAsync(host, sums, sizeof(host), cudaMemcpyDeviceToHost, s)))
        return HTD_ERR_CUDA;
    if (failed(cudaStreamSynchronize(s))) return HTD_ERR_CUDA;
    const double rr = host[0].x, ff = host[1].x;
    if (!std::isfinite(rr) || !std::isfinite(ff)) return HTD_ERR_NONFINITE;
    *rel = (ff > 0.0) ? std::sqrt(rr > 0.0 ? rr : 0.0) / std::sqrt(ff) : 0.0;
    return HTD_OK;
}
