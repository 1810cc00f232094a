// Allocation-free variant of the FP32 line sweep (sc_sweep_lines_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// sweep: code that runs while a memory pool or an allocator of another
// framework owns the device heap, real-time loops that must not block in
// cudaMalloc/cudaFree (both can synchronise the device), and embedded hosts
// that reserve all device memory up front.  This entry point takes every input
// and output buffer from the caller and keeps its only scratch -- the forward
// coherence functions parked between the two passes of each line -- in the
// file-scope array below.  The array is part of the loaded module: every GPU
// that loads the library holds its full size until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <stdint.h>

#include "riccati_step.cuh"
#include "sc.h"

namespace sc_internal {
void set_thread_error(const char *msg);  // read back through sc_last_error(NULL)
}

namespace {

// Scratch for the parked gammas: 32 MiB = 4 Mi complex floats per device.
constexpr int64_t kScratchComplex = (int64_t)4 << 20;
constexpr int kMaxDevices = 64;
constexpr int kLanes = 32;  // one warp per line, energies on the lanes
constexpr int kMaxEnergies = kLanes * 8;

static __device__ __align__(256) float2 g_noalloc_scratch[kScratchComplex];

std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

template <int EPT>
__global__ void __launch_bounds__(128) sweep_lines_static_kernel(
    const float4 *__restrict__ samples, const int32_t *__restrict__ line_slot0,
    const int32_t *__restrict__ line_ns, const float2 *__restrict__ line_len,
    const float2 *__restrict__ entry, int32_t n_lines, int32_t max_ns, int32_t n_e, float t,
    float h, float4 *__restrict__ images, float2 *__restrict__ exits, float2 *scratch, int64_t slab) {
    using scd::Cx;
    using scd::StepCoef;
    typedef Cx<float> C;
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    C *park = (C *)scratch + wid * slab;
    float zi[EPT];
    bool ev[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int n = lane + kLanes * e;
        ev[e] = n < n_e;
        zi[e] = t * ((ev[e] ? n : n_e - 1) + 0.5f);  // eps_n = t (n + 1/2)
    }
    for (int64_t L = wid; L < n_lines; L += nwarps) {
        const int ns = line_ns[L];
        if (ns < 0 || ns > max_ns) {
            // the line does not fit the slab sized from max_ns: mark its exits, skip it
#pragma unroll
            for (int e = 0; e < EPT; ++e)
                if (ev[e]) {
                    exits[(int64_t)L * n_e + lane + kLanes * e] = make_float2(__int_as_float(0x7fc00000), 0.f);
                    exits[((int64_t)n_lines + L) * n_e + lane + kLanes * e] = make_float2(__int_as_float(0x7fc00000), 0.f);
                }
            continue;
        }
        const int nsl = ns > 0 ? ns : 1;
        const float4 *li = samples + line_slot0[L];
        const float lead = line_len[L].x, tail = line_len[L].y;
        // forward: +e_par from smin
        C g[EPT];
        float4 sp = li[0];
        if (entry) {
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                const float2 v = entry[(int64_t)L * n_e + (ev[e] ? lane + kLanes * e : 0)];
                g[e].x = v.x;
                g[e].y = v.y;
            }
        } else {
            const float d2 = sp.x * sp.x + sp.y * sp.y;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                StepCoef<float> c;
                scd::step_coef<float>(sp.x, sp.y, d2, sp.z, zi[e], lead, c);
                g[e] = c.gh;
            }
        }
        float4 sq = sp;
        for (int i = 0; i <= ns; ++i) {
            const float dr = 0.5f * (sp.x + sq.x), di = 0.5f * (sp.y + sq.y), av = 0.5f * (sp.z + sq.z);
            const float ell = (i == 0) ? lead : (i == ns ? tail : h);
            const float d2 = dr * dr + di * di;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                StepCoef<float> c;
                scd::step_coef<float>(dr, di, d2, av, zi[e], ell, c);
                scd::step_apply<float>(c, g[e]);
            }
            if (i < ns) {
#pragma unroll
                for (int e = 0; e < EPT; ++e) park[(int64_t)i * kLanes * EPT + lane + kLanes * e] = g[e];
            }
            sp = sq;
            sq = li[min(i + 1, nsl - 1)];
        }
#pragma unroll
        for (int e = 0; e < EPT; ++e)
            if (ev[e]) exits[(int64_t)L * n_e + lane + kLanes * e] = make_float2(g[e].x, g[e].y);
        // backward: -e_par from smax (a -> -a)
        float4 sh = li[nsl - 1];
        if (entry) {
            const float2 *eb = entry + (int64_t)n_lines * n_e;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                const float2 v = eb[(int64_t)L * n_e + (ev[e] ? lane + kLanes * e : 0)];
                g[e].x = v.x;
                g[e].y = v.y;
            }
        } else {
            const float d2 = sh.x * sh.x + sh.y * sh.y;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                StepCoef<float> c;
                scd::step_coef<float>(sh.x, sh.y, d2, -sh.z, zi[e], tail, c);
                g[e] = c.gh;
            }
        }
        float4 slo = sh;
        for (int j = 0; j <= ns; ++j) {
            const float dr = 0.5f * (sh.x + slo.x), di = 0.5f * (sh.y + slo.y), av = 0.5f * (sh.z + slo.z);
            const float ell = (j == 0) ? tail : (j == ns ? lead : h);
            const float d2 = dr * dr + di * di;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                StepCoef<float> c;
                scd::step_coef<float>(dr, di, d2, -av, zi[e], ell, c);
                scd::step_apply<float>(c, g[e]);
            }
            if (j < ns) {
                const int q = nsl - 1 - j;
                // propagator from the parked gamma (angle p) and gamma~ = conj(g)
                float sfr = 0.f, sfi = 0.f, sg = 0.f, sFr = 0.f, sFi = 0.f;
#pragma unroll
                for (int e = 0; e < EPT; ++e) {
                    if (!ev[e]) continue;
                    const C ga = park[(int64_t)q * kLanes * EPT + lane + kLanes * e];
                    const C gb = g[e];
                    const float pr = ga.x * gb.x + ga.y * gb.y, pim = ga.y * gb.x - ga.x * gb.y;
                    const float Dr = 1.f + pr, Di = pim;
                    const float rD = scd::Mth<float>::rcp(Dr * Dr + Di * Di);
                    const float ir = Dr * rD, ii = -Di * rD;
                    sg += ii;
                    sfr += (ga.x * ir - ga.y * ii) + (gb.x * ir + gb.y * ii);
                    sfi += (ga.x * ii + ga.y * ir) + (gb.y * ir - gb.x * ii);
                    sFr += ga.x + gb.x;
                    sFi += ga.y + gb.y;
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    sfr += __shfl_xor_sync(0xffffffffu, sfr, off);
                    sfi += __shfl_xor_sync(0xffffffffu, sfi, off);
                    sg += __shfl_xor_sync(0xffffffffu, sg, off);
                    sFr += __shfl_xor_sync(0xffffffffu, sFr, off);
                    sFi += __shfl_xor_sync(0xffffffffu, sFi, off);
                }
                if (lane == 0) {
                    const float4 s = li[q];
                    images[line_slot0[L] + q] = make_float4(6.283185307179586f * sfi, -6.283185307179586f * sfr,
                                                            12.566370614359172f * sg,
                                                            2.f * (s.x * sFi - s.y * sFr));
                }
            }
            sh = slo;
            slo = li[max(nsl - 2 - j, 0)];
        }
        const int64_t ob = (int64_t)n_lines * n_e;
#pragma unroll
        for (int e = 0; e < EPT; ++e)
            if (ev[e]) exits[ob + (int64_t)L * n_e + lane + kLanes * e] = make_float2(g[e].x, g[e].y);
        __syncwarp();
    }
}

// Looks up the device address of the scratch array for the current device and
// loads every energy layout's kernel.  Runs once per device (on that device's
// first call).  Under CUDA's lazy module loading a kernel is otherwise loaded at
// its first launch, which can allocate device memory for its code and
// synchronise; querying each instantiation's attributes here moves all of that
// into the first call.
sc_status noalloc_setup(int dev, void **ptr, int *sms) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            sc_internal::set_thread_error("cudaGetSymbolAddress of the static scratch failed");
            return SC_ECUDA;
        }
        const void *kernels[8] = {(const void *)sweep_lines_static_kernel<1>, (const void *)sweep_lines_static_kernel<2>,
                                  (const void *)sweep_lines_static_kernel<3>, (const void *)sweep_lines_static_kernel<4>,
                                  (const void *)sweep_lines_static_kernel<5>, (const void *)sweep_lines_static_kernel<6>,
                                  (const void *)sweep_lines_static_kernel<7>, (const void *)sweep_lines_static_kernel<8>};
        for (const void *k : kernels) {
            cudaFuncAttributes attr;
            e = cudaFuncGetAttributes(&attr, k);
            if (e != cudaSuccess) {
                sc_internal::set_thread_error("loading the allocation-free sweep kernels failed");
                return SC_ECUDA;
            }
        }
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || n < 1) {
            sc_internal::set_thread_error("cudaDeviceGetAttribute failed");
            return SC_ECUDA;
        }
        g_sm_count[dev] = n;
        g_scratch_ptr[dev] = p;
    }
    *ptr = g_scratch_ptr[dev];
    *sms = g_sm_count[dev];
    return SC_OK;
}

}  // namespace


extern "C" sc_status sc_sweep_lines_noalloc(const float *samples, const int32_t *line_slot0,
                                            const int32_t *line_ns, const float *line_len,
                                            const float *entry, int32_t n_lines, int32_t max_ns,
                                            int32_t n_e, double t, double h, float *images,
                                            float *exits, void *stream) {
    sc_internal::set_thread_error("");
    if (!samples || !line_slot0 || !line_ns || !line_len || !images || !exits) {
        sc_internal::set_thread_error("null buffer");
        return SC_EINVAL;
    }
    if (n_lines < 1 || max_ns < 0 || n_e < 1 || !(t > 0.0) || !(h > 0.0)) {
        sc_internal::set_thread_error("need n_lines >= 1, max_ns >= 0, n_e >= 1, t > 0, h > 0");
        return SC_EINVAL;
    }
    if (n_e > kMaxEnergies) {
        sc_internal::set_thread_error("n_e exceeds 256, the most this entry point handles");
        return SC_EINVAL;
    }
    const int ept = (n_e + kLanes - 1) / kLanes;
    const int64_t slab = (int64_t)(max_ns > 0 ? max_ns : 1) * kLanes * ept;  // complex per warp
    if (slab > kScratchComplex) {
        sc_internal::set_thread_error("max_ns * 32 * ceil(n_e / 32) exceeds the 4 Mi complex-float static scratch");
        return SC_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        sc_internal::set_thread_error("no current CUDA device");
        return SC_ECUDA;
    }
    void *scratch = nullptr;
    int sms = 0;
    sc_status st = noalloc_setup(dev, &scratch, &sms);
    if (st != SC_OK) return st;
    // as many warps as the scratch holds slabs, at most 16 per SM, at most one per line;
    // every launched warp owns a whole slab inside the array
    int64_t warps = kScratchComplex / slab;
    if (warps > (int64_t)sms * 16) warps = (int64_t)sms * 16;
    if (warps > n_lines) warps = n_lines;
    const int per_block = warps >= 4 ? 4 : (int)warps;
    const int blocks = (int)(warps / per_block);
    // an error left by earlier work on this thread is not this call's: report it
    // without clearing it, and launch nothing
    if (cudaPeekAtLastError() != cudaSuccess) {
        sc_internal::set_thread_error("a CUDA error from earlier work is pending on this thread; nothing launched");
        return SC_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const float4 *sm = (const float4 *)samples;
    const float2 *len = (const float2 *)line_len;
    const float2 *en = (const float2 *)entry;
    float4 *img = (float4 *)images;
    float2 *ex = (float2 *)exits;
    float2 *scr = (float2 *)scratch;
    switch (ept) {
#define SC_CASE(E)                                                                                     \
    case E:                                                                                            \
        sweep_lines_static_kernel<E><<<blocks, 32 * per_block, 0, s>>>(sm, line_slot0, line_ns, len, en, n_lines, \
                                                             max_ns, n_e, (float)t, (float)h, img, ex, scr, slab); \
        break;
        SC_CASE(1) SC_CASE(2) SC_CASE(3) SC_CASE(4) SC_CASE(5) SC_CASE(6) SC_CASE(7) SC_CASE(8)
#undef SC_CASE
        default: sc_internal::set_thread_error("bad energy layout"); return SC_EINVAL;
    }
    const cudaError_t e = cudaGetLastError();  // this launch's own error (none was pending)
    if (e != cudaSuccess) {
        sc_internal::set_thread_error(cudaGetErrorString(e));
        return SC_ECUDA;
    }
    return SC_OK;
}

