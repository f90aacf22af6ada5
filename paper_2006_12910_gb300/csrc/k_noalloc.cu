// k_noalloc.cu -- global mass / momentum sums over caller-owned device buffers,
// with no device allocation at all.
//
// Who needs this: callers that must not allocate device memory -- code that
// runs while a stream is being captured (cudaMalloc and cudaFree are not
// allowed there and synchronise the device outside it), real-time stepping
// loops that cannot afford the implicit device synchronisation of
// cudaMalloc / cudaFree, and frameworks whose own memory pool owns the GPU
// and forbids side allocations.  They hold the populations in their own
// buffers (for example torch tensors) and want the checks without creating a
// context, which would allocate.
//
// How: the per-row partial sums live in one file-scope __device__ array of
// LBM_NOALLOC_MAX_ROWS x 3 doubles (384 KiB), which every GPU that loads this
// library keeps until the process exits.  Host code cannot use the array's
// name as a device address, so the first call on each device, with that
// device current, asks the runtime for the address (cudaGetSymbolAddress) and
// caches it; later calls reuse it.  Every slot the final sum reads is written
// earlier in the same call, so nothing has to start at zero, but all calls
// share the one array: calls whose kernels overlap on the GPU (on different
// streams, or from different threads) race on it and must be ordered.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "kernels.h"
#include "lbm_dev.cuh"

namespace lbmk {

static __device__ __align__(256) double g_noalloc_rows[3 * LBM_NOALLOC_MAX_ROWS];

constexpr int NOALLOC_MAX_DEVICES = 64;
static void* g_rows_addr[NOALLOC_MAX_DEVICES] = {};
static std::mutex g_rows_mutex;

struct NoallocArgs {
    const void* f;
    const uint8_t* solid;
    int nx, ny, pitch;
    double rho0, scale_inv;
    double* rows;
    double* out;
};

// One CTA per row (grid-stride over rows): FP64 sums of sum_i f_i, sum_i f_i e_ix,
// sum_i f_i e_iy over the fluid nodes of the row, fixed-order tree per CTA.
template <class S>
__global__ void __launch_bounds__(256) k_rows_noalloc(NoallocArgs a) {
    __shared__ double sh[3][256];
    const typename S::T* f = static_cast<const typename S::T*>(a.f);
    const int64_t plane = (int64_t)a.ny * a.pitch;
    for (int y = blockIdx.x; y < a.ny; y += gridDim.x) {
        double m = 0.0, px = 0.0, py = 0.0;
        for (int x = threadIdx.x; x < a.nx; x += blockDim.x) {
            const int64_t k = (int64_t)y * a.pitch + x;
            if (a.solid && a.solid[k]) continue;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                double v = (double)to_a(f[(int64_t)i * plane + k], (typename S::A)a.scale_inv);
                if (S::SHIFT) v += wgt(i) * a.rho0;
                m += v;
                px += v * cx(i);
                py += v * cy(i);
            }
        }
        sh[0][threadIdx.x] = m;
        sh[1][threadIdx.x] = px;
        sh[2][threadIdx.x] = py;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s)
                for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x < 3) a.rows[3 * (int64_t)y + threadIdx.x] = sh[threadIdx.x][0];
        __syncthreads();
    }
}

// Sum of the row partials in row order, one thread per component.
__global__ void k_rows_final(NoallocArgs a) {
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int y = 0; y < a.ny; ++y) s += a.rows[3 * (int64_t)y + threadIdx.x];
        a.out[threadIdx.x] = s;
    }
}

}  // namespace lbmk

namespace {
int noalloc_fail(int code, const char* msg) {
    lbmk::set_global_error(msg);
    return code;
}
int noalloc_cuda_fail(const char* what, cudaError_t e) {
    std::string m = std::string("lbm_checks_noalloc: ") + what + ": " + cudaGetErrorString(e);
    lbmk::set_global_error(m.c_str());
    return LBM_E_CUDA;
}
}  // namespace

extern "C" int lbm_checks_noalloc(const void* d_populations, int32_t store, int32_t nx, int32_t ny, int32_t pitch,
                                  double rho0, double store_scale, const uint8_t* d_solid, double* d_out3,
                                  void* cuda_stream) {
    using namespace lbmk;
    if (!d_populations || !d_out3) return noalloc_fail(LBM_E_INVAL, "lbm_checks_noalloc: NULL population or output buffer");
    if (nx < 1 || ny < 1 || pitch < nx) return noalloc_fail(LBM_E_INVAL, "lbm_checks_noalloc: need nx, ny >= 1 and pitch >= nx");
    if (ny > LBM_NOALLOC_MAX_ROWS)  // more rows than the static scratch holds
        return noalloc_fail(LBM_E_INVAL, "lbm_checks_noalloc: ny above LBM_NOALLOC_MAX_ROWS");
    if ((int64_t)pitch * ny > ((int64_t)1 << 31)) return noalloc_fail(LBM_E_INVAL, "lbm_checks_noalloc: plane above 2^31 elements");
    if (store < LBM_F64 || store > LBM_BF16S) return noalloc_fail(LBM_E_INVAL, "lbm_checks_noalloc: unknown store kind");
    const bool scaled = store == LBM_F16S || store == LBM_BF16S;
    if (scaled && !(store_scale > 0.0)) return noalloc_fail(LBM_E_INVAL, "lbm_checks_noalloc: store_scale must be > 0");

    // An error left pending by earlier work is the caller's, not this call's:
    // report it without clearing it.
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) return noalloc_cuda_fail("a CUDA error was pending before the call", pending);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_cuda_fail("cudaGetDevice", e);
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return noalloc_fail(LBM_E_CUDA, "lbm_checks_noalloc: device index above 63");
    void* rows = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_rows_mutex);
        if (!g_rows_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_rows);
            if (e != cudaSuccess || !p) return noalloc_cuda_fail("cudaGetSymbolAddress", e);
            g_rows_addr[dev] = p;
        }
        rows = g_rows_addr[dev];
    }
    NoallocArgs a;
    a.f = d_populations;
    a.solid = d_solid;
    a.nx = nx;
    a.ny = ny;
    a.pitch = pitch;
    a.rho0 = rho0;
    a.scale_inv = scaled ? 1.0 / store_scale : 1.0;
    a.rows = static_cast<double*>(rows);
    a.out = d_out3;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int grid = ny < 2048 ? ny : 2048;
    switch (store) {
        case LBM_F64: k_rows_noalloc<StF64><<<grid, 256, 0, s>>>(a); break;
        case LBM_F32: k_rows_noalloc<StF32><<<grid, 256, 0, s>>>(a); break;
        case LBM_F32S: k_rows_noalloc<StF32S><<<grid, 256, 0, s>>>(a); break;
        case LBM_F16S: k_rows_noalloc<StF16S><<<grid, 256, 0, s>>>(a); break;
        default: k_rows_noalloc<StBF16S><<<grid, 256, 0, s>>>(a); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_cuda_fail("row-sum launch", e);
    k_rows_final<<<1, 32, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_cuda_fail("final-sum launch", e);
    return LBM_OK;
}
