// Self-consistency accelerators of App. E on the device: the grid-sized vector
// work (differences, dot products, updates) in FP64; the scalar step-size logic
// runs on the host from the reduced dot products (accel_api.cpp).
#include "accel.cuh"

namespace scd {

namespace {

constexpr int kBlock = 256;

// component c of x and g at point i (Re, Im of each Delta component, then the
// two A components); false when the component does not exist there
__device__ __forceinline__ bool comp(const AccelArgs &a, int c, int64_t i, double &x, double &g) {
    const int nd = 2 * a.nc;
    if (c < nd) {
        if (!a.mask[i]) return false;
        const int64_t o = 2 * ((c >> 1) * a.npts + i) + (c & 1);
        x = a.delta[o];
        g = a.dnew[o];
        return true;
    }
    if (!a.aind || c >= nd + 2) return false;
    x = a.k2 * a.aind[2 * i + (c - nd)];
    g = a.k2 * a.anew[2 * i + (c - nd)];
    return true;
}

// Slots: 0 |dprev|^2, 1 dprev.(d - dprev), 2 |d - dprev|^2 (Barzilai-Borwein, all
// components); 3 + 3c + {0, 1, 2} = m_c.d_c, |m_c|^2, |d_c|^2 (CongAcc, component c).
// kAccelSums doubles per thread: the block reduction runs slot by slot.
__global__ void accel_partials_kernel(AccelArgs a, double *__restrict__ partials) {
    double s[kAccelSums];
#pragma unroll
    for (int k = 0; k < kAccelSums; ++k) s[k] = 0.0;
    const int64_t n = a.npts;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < kAccelComps; ++c) {
            double x, g;
            if (!comp(a, c, i, x, g)) continue;
            const double d = g - x;
            const double dp = a.dprev[c * n + i], mm = a.m[c * n + i];
            const double dd = d - dp;
            s[0] += dp * dp;
            s[1] += dp * dd;
            s[2] += dd * dd;
            s[3 + 3 * c] += mm * d;
            s[4 + 3 * c] += mm * mm;
            s[5 + 3 * c] += d * d;
        }
    }
    __shared__ double sh[kBlock / 32][kAccelSums];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kAccelSums; ++k) {
        double v = s[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sh[w][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kAccelSums) {
        double v = 0.0;
        for (int q = 0; q < kBlock / 32; ++q) v += sh[q][threadIdx.x];
        partials[(int64_t)blockIdx.x * kAccelSums + threadIdx.x] = v;
    }
}

// one thread per slot sums the block partials in block order
__global__ void accel_final_kernel(const double *__restrict__ partials, int blocks, double *__restrict__ sums) {
    const int k = threadIdx.x;
    if (k >= kAccelSums) return;
    double v = 0.0;
    for (int b = 0; b < blocks; ++b) v += partials[(int64_t)b * kAccelSums + k];
    sums[k] = v;
}

struct Steps {
    double alpha, beta, ac[kAccelComps], wc[kAccelComps];
};

__global__ void accel_update_kernel(AccelArgs a, int kind, Steps st) {
    const int64_t n = a.npts;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < kAccelComps; ++c) {
        double x, g;
        if (!comp(a, c, i, x, g)) continue;
        const double d = g - x;
        double xn;
        if (kind == 1) {
            const double v = (1.0 - st.beta) * a.v[c * n + i] + st.alpha * d;
            a.v[c * n + i] = v;
            xn = x + v;
        } else if (kind == 3) {
            const double m = st.wc[c] * a.m[c * n + i] + (1.0 - st.wc[c]) * d;
            a.m[c * n + i] = m;
            xn = x + st.ac[c] * m;
        } else {
            if (kind == 2) a.dprev[c * n + i] = d;
            xn = x + st.alpha * d;
        }
        if (c < 2 * a.nc)
            a.delta[2 * ((c >> 1) * n + i) + (c & 1)] = xn;
        else
            a.aind[2 * i + (c - 2 * a.nc)] = xn / a.k2;
    }
}

}  // namespace

int accel_reduce_blocks(int64_t npts, int sm_count) {
    const int64_t b = (npts + kBlock - 1) / kBlock;
    const int64_t cap = (int64_t)(sm_count > 0 ? sm_count : 1) * 4;
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

cudaError_t launch_accel_reduce(const AccelArgs &a, double *partials, int blocks, double *sums, cudaStream_t s) {
    accel_partials_kernel<<<blocks, kBlock, 0, s>>>(a, partials);
    accel_final_kernel<<<1, 32, 0, s>>>(partials, blocks, sums);
    return cudaGetLastError();
}

cudaError_t launch_accel_update(const AccelArgs &a, int kind, double alpha, double beta, const double *alpha_c,
                                const double *w_c, cudaStream_t s) {
    Steps st{};
    st.alpha = alpha;
    st.beta = beta;
    for (int c = 0; c < kAccelComps; ++c) {
        st.ac[c] = alpha_c ? alpha_c[c] : 0.0;
        st.wc[c] = w_c ? w_c[c] : 0.0;
    }
    const unsigned nb = (unsigned)((a.npts + kBlock - 1) / kBlock);
    accel_update_kernel<<<nb, kBlock, 0, s>>>(a, kind, st);
    return cudaGetLastError();
}

}  // namespace scd
