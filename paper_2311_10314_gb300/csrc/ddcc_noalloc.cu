// Per-phase mass reduction that allocates nothing (ddcc_phase_mass_noalloc).
//
// Some callers cannot call cudaMalloc: plugins of host applications that
// own every device byte through their own pool and forbid foreign
// allocations, and real-time loops that cannot afford the implicit device
// synchronisation an allocation brings.  For them this entry point keeps
// its scratch -- one FP64 partial sum per (phase, row) -- in a file-scope
// static device array of fixed size, so the caller only passes the
// populations and the output.
//
// The static array is shared by every call in the process on a device and
// keeps the last call's contents.  Every partial a call reads is written by
// the same call first, so nothing has to be cleared; calls that overlap on
// the GPU (on different streams, or from several host threads) race on the
// array and must be serialised by the caller.
#include <mutex>

#include "ddcc.h"

namespace {

constexpr int kNoallocMaxRows = DDCC_NOALLOC_MAX_ROWS;
constexpr int kNoallocPhases = DDCC_MAX_PHASES - 1;

// (phase, row) partial sums; 3 x 16384 doubles = 384 KiB per device.
static __device__ __align__(256) double g_noalloc_partials[kNoallocPhases * kNoallocMaxRows];

// One block per row: partial[i * ny + y] = sum_x sum_p f^i_p(x, y).
template <typename T>
__global__ void __launch_bounds__(256) k_mass_rows(const T* __restrict__ f, int nph, int nx, int ny,
                                                    long long row_stride, long long plane_stride,
                                                    double* __restrict__ partial) {
    __shared__ double red[kNoallocPhases][256];
    const int y = blockIdx.x;
    for (int i = 0; i < nph; ++i) {
        double acc = 0.0;
        for (int x = threadIdx.x; x < nx; x += blockDim.x) {
            const long long o = (long long)y * row_stride + x;
            for (int p = 0; p < 9; ++p) acc += (double)f[(long long)(i * 9 + p) * plane_stride + o];
        }
        red[i][threadIdx.x] = acc;
    }
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int i = 0; i < nph; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int i = 0; i < nph; ++i) partial[(long long)i * ny + y] = red[i][0];
}

// Sum the row partials of each phase in row order (deterministic).
__global__ void k_mass_rows_final(const double* __restrict__ partial, int nph, int ny,
                                  double* __restrict__ out) {
    const int i = threadIdx.x;
    if (i < nph) {
        double s = 0.0;
        for (int y = 0; y < ny; ++y) s += partial[(long long)i * ny + y];
        out[i] = s;
    }
}

// Device address of the static array, looked up once per device and kept
// for the life of the process (stale after a cudaDeviceReset of that device).
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_partials_addr[kMaxDevices] = {};

int partials_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DDCC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return DDCC_ERR_CUDA;
        g_partials_addr[dev] = p;
    }
    *out = g_partials_addr[dev];
    return DDCC_OK;
}

}  // namespace

extern "C" int ddcc_phase_mass_noalloc(const void* dev_populations, int precision, int nphase,
                                       int nx, int ny, int64_t row_stride, int64_t plane_stride,
                                       double* dev_out, void* cuda_stream) {
    if (!dev_populations || !dev_out) return DDCC_ERR_PARAM;
    if (precision != DDCC_FP64 && precision != DDCC_FP32) return DDCC_ERR_PARAM;
    if (nphase < 2 || nphase > DDCC_MAX_PHASES) return DDCC_ERR_PARAM;
    if (nx < 1 || ny < 1 || ny > kNoallocMaxRows) return DDCC_ERR_PARAM;   // beyond the static scratch
    if (row_stride < nx || plane_stride < row_stride * (int64_t)ny) return DDCC_ERR_PARAM;
    void* partials = nullptr;
    const int st = partials_address(&partials);
    if (st != DDCC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nph = nphase - 1;
    if (precision == DDCC_FP64)
        k_mass_rows<double><<<ny, 256, 0, s>>>(static_cast<const double*>(dev_populations), nph, nx, ny,
                                                row_stride, plane_stride, static_cast<double*>(partials));
    else
        k_mass_rows<float><<<ny, 256, 0, s>>>(static_cast<const float*>(dev_populations), nph, nx, ny,
                                               row_stride, plane_stride, static_cast<double*>(partials));
    k_mass_rows_final<<<1, 32, 0, s>>>(static_cast<const double*>(partials), nph, ny, dev_out);
    return cudaGetLastError() == cudaSuccess ? DDCC_OK : DDCC_ERR_CUDA;
}
