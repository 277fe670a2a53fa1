// asm_residual_noalloc: r = b - A x and ||r||_2 without allocating anything (the true residual
// that ends a Krylov solve, Section 2).
//
// Some callers cannot call cudaMalloc at the point where they need a residual: code running while
// a caller-owned memory pool forbids further device allocations, or code whose allocations must
// stay fixed after start-up (certified or real-time simulators).  This entry point gives them the
// true residual of an x they hold: it reads the matrix already stored in the handle and writes
// only the caller's buffers, and the block partial sums of the norm go to a fixed scratch array
// compiled into the library.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "asm2.h"
#include "asm2_internal.h"

namespace asm2 {

// Longest system the scratch array supports: one partial per 256 block rows.
constexpr int kNoAllocPartials = 16384;
constexpr long long kNoAllocMaxCells = 256LL * kNoAllocPartials;

// File-scope scratch: [0, kNoAllocPartials) block partials of sum r^2, then one arrival counter
// (as an unsigned int in the last 8-byte word).  Every GPU that loads the library holds it until
// the process exits.  Every call shares it: calls that overlap on the GPU race.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocPartials + 1] = {};

namespace {

__global__ void __launch_bounds__(256) k_residual_noalloc(const double* __restrict__ ell_val, const int* __restrict__ ell_col,
                                                          int ell_w, int rows_pad, int n_cells, const double* __restrict__ b,
                                                          const double* __restrict__ x, double* __restrict__ r,
                                                          double* __restrict__ norm, double* __restrict__ scratch) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (row < n_cells) {
        const long long rp = rows_pad;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < ell_w; w++) {
            const int c = ell_col[(long long)w * rp + row];
            const double x0 = x[3LL * c], x1 = x[3LL * c + 1], x2 = x[3LL * c + 2];
            const double* v = ell_val + (long long)w * 9 * rp + row;
            a0 += v[0] * x0 + v[rp] * x1 + v[2 * rp] * x2;
            a1 += v[3 * rp] * x0 + v[4 * rp] * x1 + v[5 * rp] * x2;
            a2 += v[6 * rp] * x0 + v[7 * rp] * x1 + v[8 * rp] * x2;
        }
        a0 = b[3LL * row] - a0;
        a1 = b[3LL * row + 1] - a1;
        a2 = b[3LL * row + 2] - a2;
        r[3LL * row] = a0;
        r[3LL * row + 1] = a1;
        r[3LL * row + 2] = a2;
        s = a0 * a0 + a1 * a1 + a2 * a2;
    }
    // block sum, then the last block to arrive adds the partials in index order (deterministic)
    __shared__ double red[256];
    __shared__ bool last;
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNoAllocPartials);
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(&scratch[i]);
    red[threadIdx.x] = t;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *norm = sqrt(red[0]);
        *counter = 0u;  // the next call starts from zero
    }
}

// Device address of the scratch array and the kernel, loaded once per device by
// noalloc_prepare() from asm_create.  The library's kernels are loaded lazily by CUDA (each .cu
// file is its own module), and loading a module or a kernel allocates device memory, so it must
// happen while the caller can still allocate: in asm_create, not in the first residual call.  In
// host code the array's name is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

double* scratch_of(int device) {
    if (device < 0 || device >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_mutex);
    return g_scratch_ptr[device];
}

}  // namespace

// Called by asm_create with `device` current.  The array needs no clearing: it is
// zero-initialised when its module loads, and every call leaves the counter at zero.
int noalloc_prepare(int device) {
    if (device < 0 || device >= kMaxDevices) return ASM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_ptr[device]) return ASM_OK;
    void* p = nullptr;
    cudaFuncAttributes attr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess ||
        cudaFuncGetAttributes(&attr, k_residual_noalloc) != cudaSuccess) {
        cudaGetLastError();
        return ASM_ERR_CUDA;
    }
    g_scratch_ptr[device] = static_cast<double*>(p);
    return ASM_OK;
}

}  // namespace asm2

extern "C" int asm_residual_noalloc(asm_handle h, const double* b, const double* x, double* r, double* norm) {
    using namespace asm2;
    if (!h || !b || !x || !r || !norm) return ASM_ERR_INVALID_ARG;
    MatrixView mv;
    int st = handle_matrix_view(h, &mv);
    if (st != ASM_OK) return st;
    if (mv.n_cells > kNoAllocMaxCells) return ASM_ERR_INVALID_ARG;  // beyond the scratch array
    // r is written while other threads still read x at neighbouring rows: they must not overlap
    // (r may be b: each row reads its b entries before writing the same r entries)
    const size_t n3 = 3 * (size_t)mv.n_cells;
    const uintptr_t xs = reinterpret_cast<uintptr_t>(x), rs = reinterpret_cast<uintptr_t>(r);
    if (rs < xs + n3 * sizeof(double) && xs < rs + n3 * sizeof(double)) return ASM_ERR_INVALID_ARG;
    double* scratch = scratch_of(mv.device);
    if (!scratch) return ASM_ERR_STATE;  // asm_create did not prepare this device
    if (cudaSetDevice(mv.device) != cudaSuccess) {
        cudaGetLastError();
        return ASM_ERR_CUDA;
    }
    const int blocks = (mv.n_cells + 255) / 256;
    k_residual_noalloc<<<blocks, 256, 0, mv.stream>>>(mv.ell_val, mv.ell_col, mv.ell_w, mv.rows_pad, mv.n_cells, b, x,
                                                      r, norm, scratch);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(mv.stream) != cudaSuccess) {
        cudaGetLastError();
        return ASM_ERR_CUDA;
    }
    return ASM_OK;
}
