// Batched transpose of complex samples for the multi-GPU separable 2-D
// transform: in [batch][rows][cols][vec] -> out [batch][cols][rows][vec].
// vec = 1: 32 x 32 tiles through shared memory (padded by one slot), so the
// reads and the writes are both coalesced; vec > 1: every (row, col) vector
// is copied whole by one warp (coalesced along vec).
#include "xft_common.cuh"

namespace {

template <class R>
__global__ void k_transpose_tile(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
                                 int64_t rows, int64_t cols) {
    __shared__ cpx<R> tile[32][33];
    const int64_t b = blockIdx.z;
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    const cpx<R>* src = in + b * rows * cols;
    cpx<R>* dst = out + b * rows * cols;
    const int tx = threadIdx.x, ty = threadIdx.y;          // 32 x 8 threads
    for (int k = ty; k < 32; k += 8) {
        const int64_t r = r0 + k, c = c0 + tx;
        if (r < rows && c < cols) tile[k][tx] = src[r * cols + c];
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int64_t c = c0 + k, r = r0 + tx;
        if (r < rows && c < cols) dst[c * rows + r] = tile[tx][k];
    }
}

template <class R>
__global__ void k_transpose_vec(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
                                int64_t rows, int64_t cols, int64_t vec, int64_t total) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = w0; w < total; w += nw) {          // w = (b, r, c) of the input
        const int64_t c = w % cols, r = (w / cols) % rows, b = w / (cols * rows);
        const cpx<R>* s = in + w * vec;
        cpx<R>* d = out + ((b * cols + c) * rows + r) * vec;
        for (int64_t e = lane; e < vec; e += 32) d[e] = s[e];
    }
}

template <class R>
cudaError_t launch_t(const void* in, void* out, int64_t rows, int64_t cols, int64_t vec,
                     int64_t batch, cudaStream_t stream) {
    if (vec == 1) {
        const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32), (unsigned)batch);
        if ((cols + 31) / 32 > 0x7fffffff || (rows + 31) / 32 > 65535 || batch > 65535)
            return cudaErrorInvalidConfiguration;
        k_transpose_tile<R><<<grid, dim3(32, 8), 0, stream>>>((const cpx<R>*)in, (cpx<R>*)out, rows, cols);
    } else {
        const int64_t total = batch * rows * cols;
        const int64_t blocks = (total * 32 + 255) / 256;
        k_transpose_vec<R><<<(unsigned)(blocks < 152 * 32 ? blocks : 152 * 32), 256, 0, stream>>>(
            (const cpx<R>*)in, (cpx<R>*)out, rows, cols, vec, total);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t lct_launch_transpose(int dtype, const void* in, void* out, int64_t rows, int64_t cols,
                                 int64_t vec, int64_t batch, cudaStream_t stream) {
    if (dtype == 0) return launch_t<float>(in, out, rows, cols, vec, batch, stream);
    return launch_t<double>(in, out, rows, cols, vec, batch, stream);
}
