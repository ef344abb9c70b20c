// lbib_mesh_measures_noalloc (include/lbib.h): the enclosed volume and the
// surface area of a closed triangle mesh held in device memory, computed
// without allocating anything.
//
// It is a stand-alone variant of the membrane-volume reduction that the MLS
// kernel performs every step (per-block partial sums in global scratch, then
// a fixed-order sum in the last block to finish).  Where that kernel's
// scratch belongs to a context, this one lives in a file-scope device array:
// callers that cannot call cudaMalloc can still use it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/lbib.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = LBIB_NOALLOC_MAX_TRIS / kThreads;
static_assert(LBIB_NOALLOC_MAX_TRIS % kThreads == 0, "one block per 256 triangles");
constexpr size_t kPartBytes = sizeof(double) * 2 * kMaxBlocks;  // (volume, area) per block: 64 KiB
constexpr size_t kScratchBytes = kPartBytes + 256;               // + block counter and bad-index flag

// Shared by every call on a device and kept until the process exits.  In
// host code this name is only a stand-in for the symbol: the device address
// comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_mesh_scratch[kScratchBytes];

// Device address of g_mesh_scratch in the current context.  Looked up on
// every call, never cached: a cached address would outlive a
// cudaDeviceReset or any re-creation of the device's primary context.  The
// lookup allocates nothing; only the first one in a process may load the
// module (lazy loading), which is why the first call must precede any
// stream capture.
cudaError_t scratch_address(unsigned char **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_mesh_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char *>(p);
    return cudaSuccess;
}

// One thread per triangle: X0 . (X1 x X2) (six times the signed volume of
// the tetrahedron it spans with the origin) and |(X1 - X0) x (X2 - X0)|
// (twice its area).  Blocks reduce in shared memory in a fixed order and
// write one partial each; the last block to finish sums the partials in a
// fixed order, so the result does not depend on block scheduling.
__global__ void __launch_bounds__(kThreads) k_mesh_measures(const double *__restrict__ X, int nv,
                                                           const int *__restrict__ tri, int nt,
                                                           double *__restrict__ out,
                                                           unsigned char *__restrict__ scratch) {
    double *part = reinterpret_cast<double *>(scratch);
    unsigned int *count = reinterpret_cast<unsigned int *>(scratch + kPartBytes);
    unsigned int *bad = count + 1;
    __shared__ double sv[kThreads], sa[kThreads];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const int t = blockIdx.x * kThreads + tid;
    double v = 0.0, a = 0.0;
    if (t < nt) {
        const int i0 = tri[3 * t], i1 = tri[3 * t + 1], i2 = tri[3 * t + 2];
        if (i0 < 0 || i0 >= nv || i1 < 0 || i1 >= nv || i2 < 0 || i2 >= nv) {
            atomicOr(bad, 1u);  // skip the access, poison the result
        } else {
            const double x0 = X[3 * i0], y0 = X[3 * i0 + 1], z0 = X[3 * i0 + 2];
            const double x1 = X[3 * i1], y1 = X[3 * i1 + 1], z1 = X[3 * i1 + 2];
            const double x2 = X[3 * i2], y2 = X[3 * i2 + 1], z2 = X[3 * i2 + 2];
            v = x0 * (y1 * z2 - z1 * y2) + y0 * (z1 * x2 - x1 * z2) + z0 * (x1 * y2 - y1 * x2);
            const double ex = x1 - x0, ey = y1 - y0, ez = z1 - z0;
            const double fx = x2 - x0, fy = y2 - y0, fz = z2 - z0;
            const double nx = ey * fz - ez * fy, ny = ez * fx - ex * fz, nz = ex * fy - ey * fx;
            a = sqrt(nx * nx + ny * ny + nz * nz);
        }
    }
    sv[tid] = v;
    sa[tid] = a;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (tid < s) {
            sv[tid] += sv[tid + s];
            sa[tid] += sa[tid + s];
        }
        __syncthreads();
    }
    if (tid == 0) {
        part[2 * blockIdx.x] = sv[0];
        part[2 * blockIdx.x + 1] = sa[0];
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    v = 0.0;
    a = 0.0;
    for (int b = tid; b < (int)gridDim.x; b += kThreads) {
        v += __ldcg(part + 2 * b);
        a += __ldcg(part + 2 * b + 1);
    }
    sv[tid] = v;
    sa[tid] = a;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (tid < s) {
            sv[tid] += sv[tid + s];
            sa[tid] += sa[tid + s];
        }
        __syncthreads();
    }
    if (tid == 0) {
        const bool poisoned = __ldcg(bad) != 0u;
        out[0] = poisoned ? nan("") : sv[0] / 6.0;
        out[1] = poisoned ? nan("") : 0.5 * sa[0];
    }
}

}  // namespace

extern "C" int lbib_mesh_measures_noalloc(const double *X, int nv, const int *tris, int nt, double *out,
                                          void *stream) {
    if (nt > LBIB_NOALLOC_MAX_TRIS) return LBIB_ETOOBIG;
    if (nt < 0 || nv < 0 || nv > INT32_MAX / 3 || !out || (nt > 0 && (!X || !tris))) return LBIB_EINVAL;
    unsigned char *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return LBIB_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the block counter and the bad-index flag must start at zero; the
    // partials are overwritten before they are read
    e = cudaMemsetAsync(scratch + kPartBytes, 0, 2 * sizeof(unsigned int), s);
    if (e != cudaSuccess) return LBIB_ECUDA;
    const int blocks = nt > 0 ? (nt + kThreads - 1) / kThreads : 1;
    k_mesh_measures<<<blocks, kThreads, 0, s>>>(X, nv, tris, nt, out, scratch);
    e = cudaGetLastError();
    return e == cudaSuccess ? LBIB_OK : LBIB_ECUDA;
}
