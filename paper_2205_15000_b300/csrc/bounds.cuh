// Index checks of the bounds-checked build.
//
// Compiled with -DSC_DEBUG_BOUNDS (the library libsc_checked.so), every index
// the kernels take from a table -- line, line group, image slot, sample, exit
// slot of a boundary link, slab row of the parked coherence functions, padded
// grid point, rotate-back record -- is compared with the size of the table it
// indexes before the access.  A failed check skips the access (a load yields
// zero) and counts one violation in a device counter of its translation unit;
// sc_debug_bounds sums the counters.  In the regular build the checks compile
// to nothing.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace scd {

#if defined(SC_DEBUG_BOUNDS) && defined(__CUDACC__)
static __device__ unsigned long long g_bounds_bad;  // one counter per translation unit
__device__ __forceinline__ bool in_bounds(int64_t i, int64_t n) {
    if (i >= 0 && i < n) return true;
    atomicAdd(&g_bounds_bad, 1ull);
    return false;
}
// the counter of the including translation unit: read, and reset to zero if asked
#define SC_BOUNDS_ACCESSOR(fn)                                                             \
    cudaError_t fn(unsigned long long *v, bool reset) {                                    \
        cudaError_t e = cudaMemcpyFromSymbol(v, g_bounds_bad, sizeof(unsigned long long)); \
        if (e == cudaSuccess && reset) {                                                   \
            const unsigned long long z = 0;                                                \
            e = cudaMemcpyToSymbol(g_bounds_bad, &z, sizeof z);                            \
        }                                                                                  \
        return e;                                                                          \
    }
#else
__device__ __forceinline__ constexpr bool in_bounds(int64_t, int64_t) { return true; }
#define SC_BOUNDS_ACCESSOR(fn)                               \
    cudaError_t fn(unsigned long long *v, bool) {            \
        *v = 0;                                              \
        return cudaSuccess;                                  \
    }
#endif

// checked load: t[i] if 0 <= i < n, else a zero value (and a violation)
template <typename T>
__device__ __forceinline__ T ld_chk(const T *t, int64_t i, int64_t n) {
    return in_bounds(i, n) ? t[i] : T{};
}

// the per-unit accessors (sweep_f32.cu, sweep_side_f32.cu, sweep_f64.cu, adjoint_f32.cu,
// adjoint_f64.cu, adjoint.cu, lattice_f32.cu, kernels.cu)
cudaError_t bounds_sweep_f32(unsigned long long *v, bool reset);
cudaError_t bounds_sweep_side_f32(unsigned long long *v, bool reset);
cudaError_t bounds_sweep_f64(unsigned long long *v, bool reset);
cudaError_t bounds_adjoint_f32(unsigned long long *v, bool reset);
cudaError_t bounds_adjoint_f64(unsigned long long *v, bool reset);
cudaError_t bounds_adjoint_transposes(unsigned long long *v, bool reset);
cudaError_t bounds_lattice_f32(unsigned long long *v, bool reset);
cudaError_t bounds_kernels(unsigned long long *v, bool reset);

}  // namespace scd

namespace scd {

// The tables one line of a sweep reads and writes: its image slots, its exit
// slots, its entry taps (when the sweep starts from the previous exits) and its
// rows of the warp's slab (slab_first: the line's first slab element from the
// start of the scratch; slab_len: elements per sample row).  False, with the
// violation counted, when one of them is out of range.
template <typename LD>
__device__ __forceinline__ bool line_tables_ok(const LD &ln, int64_t n_slots, int32_t n_lines, bool taps,
                                               int64_t slab_first, int64_t slab_len, int64_t scratch_elems) {
    const int64_t nsl = ln.ns > 0 ? ln.ns : 1, rows = 2 * (int64_t)n_lines;
    bool ok = in_bounds(ln.slot0, n_slots) && in_bounds(ln.slot0 + nsl - 1, n_slots);
    ok = ok && in_bounds(ln.exit_f, rows) && in_bounds(ln.exit_b, rows);
    if (taps)
        for (int q = 0; q < 4; ++q) ok = ok && in_bounds(ln.tap_f[q], rows) && in_bounds(ln.tap_b[q], rows);
    return ok && in_bounds(slab_first, scratch_elems) && in_bounds(slab_first + nsl * slab_len - 1, scratch_elems);
}

}  // namespace scd
