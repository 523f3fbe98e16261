// skel_direct_noalloc: the direct sum u = A q (FP64, complex128 for
// Helmholtz) on caller-owned device buffers, with no device allocation at all.
//
// It is the plan-free form of the translation kernel's scheme: one warp owns
// 32 targets and one block of sources, writes its partial sums to scratch
// memory, and a second kernel adds the partial sums of each target in a fixed
// order. Here the scratch is a file-scope __device__ array of fixed size
// instead of memory owned by a plan, so the call works for callers that
// cannot allocate device memory: code that runs inside a framework which owns
// (and has reserved) the device memory pool, or a loop that must not take the
// device-wide synchronisation a cudaMalloc / cudaFree can cause.
//
// Rules of use (also in include/skel.h):
//   * The array takes kStaticScratchBytes of device memory on every GPU where
//     the library is loaded, until the process exits.
//   * The first call on a device looks up the array's device address on
//     that device (cudaGetSymbolAddress); make that first call before any
//     stream capture.
//   * All calls share the array, on every stream: calls that overlap on the
//     GPU race on it. Each call overwrites every scratch value it later reads,
//     so nothing has to start at zero.
//   * Problems whose partial sums do not fit are rejected with SKEL_ERR_ARG.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/skel.h"
#include "host.h"

namespace skel {

namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // 32 MiB
constexpr int kNaWarps = 8;                                 // warps per CTA
constexpr int kNaSrcBlock = 4096;                           // sources per warp work item

static __device__ __align__(256) unsigned char g_noalloc_scratch[kStaticScratchBytes];

std::mutex g_mu;
std::vector<void*> g_addr;                                  // per device: the array's device address

// Green's function without the 1/(4 pi) or -1/(4 pi) factor; zero at r = 0
template <int KIND>
__device__ __forceinline__ void na_green(double r2, double kappa, double& gr, double& gi) {
    gr = 0.0;
    gi = 0.0;
    if (!(r2 > 0.0)) return;
    if (KIND == 0) {
        gr = log(r2);
    } else if (KIND == 1) {
        gr = rsqrt(r2);
    } else if (KIND == 3) {
        const double kr = kappa * sqrt(r2);
        gr = -y0(kr);
        gi = j0(kr);
    } else {
        const double ri = rsqrt(r2);
        double s, c;
        sincos(kappa * r2 * ri, &s, &c);
        gr = c * ri;
        gi = s * ri;
    }
}

// warp item = (32-target chunk, source block): partial sum of right-hand side r
template <int KIND>
__global__ void __launch_bounds__(kNaWarps * 32)
na_partial_kernel(const double* __restrict__ x, int64_t n, int dim, const double* __restrict__ q, int r,
                  double kappa, double* __restrict__ part, int64_t nblk, int64_t nitems) {
    constexpr int W = (KIND == 2 || KIND == 3) ? 2 : 1;    // doubles per charge
    __shared__ double sx[kNaWarps][32][4 + W];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kNaWarps + warp;
    if (item >= nitems) return;
    const int64_t chunk = item / nblk, blk = item % nblk;
    const int64_t i = chunk * 32 + lane;
    double tx[3] = {0.0, 0.0, 0.0};
    if (i < n)
        for (int d = 0; d < dim; ++d) tx[d] = x[i * dim + d];
    double ar = 0.0, ai = 0.0;
    const int64_t s0 = blk * kNaSrcBlock, s1 = min(n, s0 + kNaSrcBlock);
    for (int64_t b = s0; b < s1; b += 32) {
        const int cnt = (int)min((int64_t)32, s1 - b);
        if (lane < cnt) {
            const int64_t j = b + lane;
            for (int d = 0; d < 3; ++d) sx[warp][lane][d] = d < dim ? x[j * dim + d] : 0.0;
            for (int w = 0; w < W; ++w) sx[warp][lane][4 + w] = q[((int64_t)r * n + j) * W + w];
        }
        __syncwarp();
        for (int jj = 0; jj < cnt; ++jj) {
            const double dx = tx[0] - sx[warp][jj][0], dy = tx[1] - sx[warp][jj][1], dz = tx[2] - sx[warp][jj][2];
            double gr, gi;
            na_green<KIND>(dx * dx + dy * dy + dz * dz, kappa, gr, gi);
            if (W == 2) {
                const double qr = sx[warp][jj][4], qi = sx[warp][jj][5];
                ar += gr * qr - gi * qi;
                ai += gr * qi + gi * qr;
            } else {
                ar += gr * sx[warp][jj][4];
            }
        }
        __syncwarp();
    }
    part[(item * 32 + lane) * W] = ar;
    if (W == 2) part[(item * 32 + lane) * W + 1] = ai;
}

// u_i (right-hand side r) = scale * sum over source blocks, in block order
template <int W>
__global__ void na_reduce_kernel(const double* __restrict__ part, int64_t n, int64_t nblk, int r, double scale,
                                 double* __restrict__ u) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t chunk = i / 32, lane = i % 32;
    for (int w = 0; w < W; ++w) {
        double s = 0.0;
        for (int64_t blk = 0; blk < nblk; ++blk) s += part[((chunk * nblk + blk) * 32 + lane) * W + w];
        u[((int64_t)r * n + i) * W + w] = scale * s;
    }
}

}  // namespace

}  // namespace skel

extern "C" int skel_direct_noalloc(const double* points, int64_t n, int dim, skel_kernel k, const double* q,
                                   double* u, int nrhs, void* stream) {
    using namespace skel;
    if (!points || !q || !u) return set_error(SKEL_ERR_ARG, "NULL argument");
    if (n < 1 || nrhs < 1) return set_error(SKEL_ERR_ARG, "n and nrhs must be >= 1");
    {
        const std::string m = kernel_args_error(k.kind, k.kappa, dim);   // the rules skel_build applies
        if (!m.empty()) return set_error(SKEL_ERR_ARG, m);
    }
    const int W = (k.kind == SKEL_HELMHOLTZ_3D || k.kind == SKEL_HELMHOLTZ_2D) ? 2 : 1;
    const int64_t nchunk = (n + 31) / 32, nblk = (n + kNaSrcBlock - 1) / kNaSrcBlock;
    const int64_t nitems = nchunk * nblk;
    if ((double)nitems * 32.0 * W * sizeof(double) > (double)kStaticScratchBytes)
        return set_error(SKEL_ERR_ARG, "problem too large for the static scratch array (" +
                                           std::to_string(kStaticScratchBytes >> 20) + " MiB of partial sums)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return set_error(SKEL_ERR_CUDA, "cudaGetDevice failed");
    }
    if (pointer_place(points, dev) != 1 || pointer_place(q, dev) != 1 || pointer_place(u, dev) != 1)
        return set_error(SKEL_ERR_ARG, "points, q and u must be device pointers of the current device");
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if ((int)g_addr.size() <= dev) g_addr.resize(dev + 1, nullptr);
        if (!g_addr[dev]) {
            // the host-side name of the array is not a device address: look it up on this device
            cudaError_t e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_addr[dev] = nullptr;
                return set_error(SKEL_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
        }
        scratch = g_addr[dev];
    }
    double* part = static_cast<double*>(scratch);
    cudaStream_t st = (cudaStream_t)stream;
    const double pi = 3.14159265358979323846;
    const double scale = k.kind == SKEL_LAPLACE_2D ? -1.0 / (4.0 * pi) : k.kind == SKEL_HELMHOLTZ_2D ? 0.25 : 1.0 / (4.0 * pi);
    const unsigned grid = (unsigned)((nitems + kNaWarps - 1) / kNaWarps);
    // an error left pending by the caller's earlier work is reported as such
    // (and cleared) before this call launches anything of its own
    {
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return set_error(SKEL_ERR_CUDA, std::string("an earlier CUDA error was pending: ") + cudaGetErrorString(e));
    }
    for (int r = 0; r < nrhs; ++r) {
        if (k.kind == SKEL_LAPLACE_2D)
            na_partial_kernel<0><<<grid, kNaWarps * 32, 0, st>>>(points, n, dim, q, r, k.kappa, part, nblk, nitems);
        else if (k.kind == SKEL_LAPLACE_3D)
            na_partial_kernel<1><<<grid, kNaWarps * 32, 0, st>>>(points, n, dim, q, r, k.kappa, part, nblk, nitems);
        else if (k.kind == SKEL_HELMHOLTZ_3D)
            na_partial_kernel<2><<<grid, kNaWarps * 32, 0, st>>>(points, n, dim, q, r, k.kappa, part, nblk, nitems);
        else
            na_partial_kernel<3><<<grid, kNaWarps * 32, 0, st>>>(points, n, dim, q, r, k.kappa, part, nblk, nitems);
        if (W == 2) na_reduce_kernel<2><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, n, nblk, r, scale, u);
        else na_reduce_kernel<1><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, n, nblk, r, scale, u);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return set_error(SKEL_ERR_CUDA, std::string("launch of this call's kernels (right-hand side ") +
                                                std::to_string(r) + "): " + cudaGetErrorString(e));
    }
    return SKEL_OK;
}
