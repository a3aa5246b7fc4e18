// Row copies for a decomposition of the grid into y slabs (ddcc_get_rows,
// ddcc_set_rows): rows [y0, y0 + n) of the population planes and the lagged
// planes, x in [0, nx), to or from a dense buffer laid out [plane][row][x].
#include "ddcc_internal.h"

namespace ddcc {
namespace {

inline int copy_blocks(long long n) {
    const long long b = (n + 255) / 256;
    return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

template <typename T>
__global__ void k_rows_copy(T* __restrict__ pop, T* __restrict__ lag, int npop, int nlag, KParams<T> P, int y0,
                            int n, T* __restrict__ buf, int to_buf) {
    const long long per = (long long)n * P.nx;
    const long long total = per * (npop + nlag);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i / per);
        const long long rem = i - q * per;
        const int r = (int)(rem / P.nx), x = (int)(rem - (long long)r * P.nx);
        T* plane = q < npop ? pop + (long long)q * P.plane : lag + (long long)(q - npop) * P.plane;
        T& node = plane[P.org + (long long)(y0 + r) * P.pitch + x];
        if (to_buf) buf[i] = node;
        else node = buf[i];
    }
}

}  // namespace

template <typename T>
cudaError_t launch_rows_copy(T* pop, T* lag, int npop, int nlag, const KParams<T>& kp, int y0, int n, T* buf,
                             int to_buf, cudaStream_t s) {
    k_rows_copy<T><<<copy_blocks((long long)n * kp.nx * (npop + nlag)), 256, 0, s>>>(pop, lag, npop, nlag, kp, y0, n,
                                                                                     buf, to_buf);
    return cudaGetLastError();
}
template cudaError_t launch_rows_copy<float>(float*, float*, int, int, const KParams<float>&, int, int, float*, int,
                                             cudaStream_t);
template cudaError_t launch_rows_copy<double>(double*, double*, int, int, const KParams<double>&, int, int, double*,
                                              int, cudaStream_t);

}  // namespace ddcc
