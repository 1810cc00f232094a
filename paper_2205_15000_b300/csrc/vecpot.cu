// Induced vector potential by zero-padded FFT convolution (App. D):
//   A_ind(R_i) = -(1/kappa^2) sum_k G(R_i - R_k) (j_k - <j>)
// with G the cell-integrated Green's function of the 2D Laplacian.  G is real
// and even, so both components are convolved at once as the complex field
// (j_x - <j_x>) + i (j_y - <j_y>).  The grid is padded to Px x Py (powers of
// two >= 2 nx, 2 ny), which makes the circular convolution the linear one on
// the grid; the transform of the wrapped G table is computed once.
//
// 2D FFT: one radix-2 transform per row in shared memory (bit-reversed load,
// log2 n butterfly stages with a twiddle table), a tiled transpose, the row
// transforms of the transposed array (the columns), and the product with the
// kernel's transform in that transposed layout; the inverse runs the same
// steps backwards.  FP64 throughout.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "vecpot.cuh"

namespace scd {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// one block per row of n = 2^logn complex values; tw[k] = exp(-2 pi i k / n), k < n/2
__global__ void fft_rows_kernel(double2 *__restrict__ data, int logn, const double2 *__restrict__ tw,
                                int inverse) {
    extern __shared__ double2 sm[];
    const int n = 1 << logn;
    double2 *row = data + (int64_t)blockIdx.x * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) sm[__brev((unsigned)i) >> (32 - logn)] = row[i];
    for (int s = 1; s <= logn; ++s) {
        __syncthreads();
        const int half = 1 << (s - 1), stride = n >> s;  // twiddle step for this stage
        for (int t = threadIdx.x; t < n / 2; t += blockDim.x) {
            const int pos = t & (half - 1);
            const int i = ((t >> (s - 1)) << s) + pos, j = i + half;
            double2 w = tw[pos * stride];
            if (inverse) w.y = -w.y;
            const double2 u = sm[i], v = cmul(sm[j], w);
            sm[i] = make_double2(u.x + v.x, u.y + v.y);
            sm[j] = make_double2(u.x - v.x, u.y - v.y);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) row[i] = sm[i];
}

// out[c][r] = in[r][c] for an rows x cols array, 32 x 32 tiles
__global__ void transpose_kernel(const double2 *__restrict__ in, double2 *__restrict__ out, int rows, int cols) {
    __shared__ double2 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = in[(int64_t)r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(int64_t)c * rows + r] = tile[threadIdx.x][k];
    }
}

// padded source: (j - <j>) on grain points, zero elsewhere
__global__ void vp_pack_kernel(GridDev grid, const uint8_t *__restrict__ mask, const double *__restrict__ j,
                               const double *__restrict__ jsum, double n_in, int px, int py,
                               double2 *__restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)px * py) return;
    const int x = (int)(q % px), y = (int)(q / px);
    double2 v = make_double2(0.0, 0.0);
    if (x < grid.nx && y < grid.ny) {
        const int64_t i = (int64_t)y * grid.nx + x;
        if (mask[i]) v = make_double2(j[2 * i] - jsum[0] / n_in, j[2 * i + 1] - jsum[1] / n_in);
    }
    out[q] = v;
}

// wrapped kernel table: G(|dx|, |dy|) at every padded offset within the grid's reach
__global__ void vp_kernel_pack(const double *__restrict__ G, int W, int nx, int ny, int px, int py,
                               double2 *__restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)px * py) return;
    const int x = (int)(q % px), y = (int)(q / px);
    const int dx = x < nx ? x : (x > px - nx ? px - x : -1);
    const int dy = y < ny ? y : (y > py - ny ? py - y : -1);
    out[q] = make_double2(dx >= 0 && dy >= 0 ? G[(int64_t)dx * W + dy] : 0.0, 0.0);
}

__global__ void vp_mul_kernel(double2 *__restrict__ a, const double2 *__restrict__ b, int64_t n) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) a[q] = cmul(a[q], b[q]);
}

__global__ void vp_unpack_kernel(const double2 *__restrict__ in, int px, int nx, int ny, double scale,
                                 double *__restrict__ aind) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nx * ny) return;
    const int x = (int)(i % nx), y = (int)(i / nx);
    const double2 v = in[(int64_t)y * px + x];
    aind[2 * i] = scale * v.x;
    aind[2 * i + 1] = scale * v.y;
}

cudaError_t rows(double2 *d, int n_rows, int logn, const double2 *tw, bool inverse, cudaStream_t st) {
    if (n_rows <= 0) return cudaSuccess;
    const int n = 1 << logn;
    const int bs = n / 2 < 512 ? n / 2 : 512;
    fft_rows_kernel<<<n_rows, bs, n * sizeof(double2), st>>>(d, logn, tw, inverse ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t transpose(const double2 *in, double2 *out, int r, int c, cudaStream_t st) {
    dim3 grid((c + 31) / 32, (r + 31) / 32), block(32, 8);
    transpose_kernel<<<grid, block, 0, st>>>(in, out, r, c);
    return cudaGetLastError();
}

}  // namespace

int vecpot_fft_log2(int n_grid) {
    int l = 1;
    while ((1 << l) < 2 * n_grid) ++l;
    return l;
}

cudaError_t vecpot_fft_attributes() {
    return cudaFuncSetAttribute(fft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kVecpotMaxFft * sizeof(double2)));
}

// forward 2D transform of buf (py x px, first `live_rows` rows non-zero) into
// tbuf (px x py, transposed)
static cudaError_t forward2d(const VecpotFft &f, int live_rows, cudaStream_t st) {
    cudaError_t e = rows(f.buf, live_rows, f.lx, f.tw_x, false, st);
    if (e == cudaSuccess) e = transpose(f.buf, f.tbuf, f.py, f.px, st);
    if (e == cudaSuccess) e = rows(f.tbuf, f.px, f.ly, f.tw_y, false, st);
    return e;
}

cudaError_t vecpot_fft_prepare(const VecpotFft &f, const double *G, int W, int nx, int ny, cudaStream_t st) {
    const int64_t n = (int64_t)f.px * f.py;
    const int bs = 256;
    vp_kernel_pack<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(G, W, nx, ny, f.px, f.py, f.buf);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = forward2d(f, f.py, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f.ghat, f.tbuf, n * sizeof(double2), cudaMemcpyDeviceToDevice, st);
    return e;
}

cudaError_t vecpot_fft_apply(const VecpotFft &f, const GridDev &grid, const uint8_t *mask, const double *j,
                             const double *jsum, double n_in, double inv_k2, double *aind, cudaStream_t st) {
    const int64_t n = (int64_t)f.px * f.py;
    const int bs = 256;
    vp_pack_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(grid, mask, j, jsum, n_in, f.px, f.py, f.buf);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = forward2d(f, grid.ny, st);
    if (e == cudaSuccess) {
        vp_mul_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(f.tbuf, f.ghat, n);
        e = cudaGetLastError();
    }
    // inverse: columns (rows of the transposed array), transpose back, then the
    // rows that hold grid points
    if (e == cudaSuccess) e = rows(f.tbuf, f.px, f.ly, f.tw_y, true, st);
    if (e == cudaSuccess) e = transpose(f.tbuf, f.buf, f.px, f.py, st);
    if (e == cudaSuccess) e = rows(f.buf, grid.ny, f.lx, f.tw_x, true, st);
    if (e == cudaSuccess) {
        const int64_t np = (int64_t)grid.nx * grid.ny;
        vp_unpack_kernel<<<(unsigned)((np + bs - 1) / bs), bs, 0, st>>>(f.buf, f.px, grid.nx, grid.ny,
                                                                        -inv_k2 / (double)n, aind);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace scd
