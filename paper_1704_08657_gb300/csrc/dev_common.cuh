// dev_common.cuh -- device building blocks shared by the libdwt2 kernels:
// inline-PTX wrappers for mbarriers and TMA (cp.async.bulk.tensor), bounded
// waits that report a timeout instead of hanging, the per-lane quad-row
// register type, warp shuffles, index folding and guarded stores.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace dwt2 {

constexpr unsigned FULL = 0xffffffffu;

// ----------------------------------------------------------------- geometry
// A warp owns a strip of 32*QL quads (64*QL pixels) per quad row: lane l
// holds the quads QL*l .. QL*l+QL-1 of the strip.  Two quads on each side are
// halo: after the lifting steps only the inner 32*QL-4 quads are exact, so a
// strip outputs that many quads and neighbouring strips overlap by 8 pixels.
constexpr int HALO_Q = 2;  // halo quads on each side

// whole-sample symmetric index fold for any integer k and n >= 2:
// ... 2 1 | 0 1 2 ... n-1 | n-2 n-3 ...
__device__ __forceinline__ int fold_ws(int k, int n) {
    const int per = 2 * (n - 1);
    int m = k % per;
    if (m < 0) m += per;
    return m < n ? m : per - m;
}

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// one arrival (release semantics at CTA scope)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar`, giving up after `limit_ns`.  On expiry the
// device status word gets DEV_TIMEOUT and false is returned; every lane of the
// warp agrees on the result.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned* status,
                                                  uint64_t limit_ns) {
    bool ok = mbar_try_wait(bar, parity);
    if (!ok) {
        const uint64_t t0 = globaltimer_ns();
        while (!(ok = mbar_try_wait(bar, parity))) {
            if (globaltimer_ns() - t0 > limit_ns) break;
        }
    }
    ok = __all_sync(FULL, ok);
    if (!ok && (threadIdx.x & 31) == 0 && status) atomicOr(status, DEV_TIMEOUT);
    return ok;
}

// ------------------------------------------------- checked build (DWT2_CHECKED)
// Range checks standing in for a memory checker: compiled with DWT2_CHECKED,
// every global access of the transform kernels and every shared-memory index
// computed at run time is tested against the extent of its buffer first; a
// violation sets DEV_CHECK in the status word (dwt2_status then reports
// DWT2_ERR_DEVICE_CHECK), the access is skipped (a load reads element 0 of its
// buffer instead, so that no wait is left without its copy) and the kernel
// stops at the end of the unit.  In normal builds every check is `true` and
// compiles away.
#ifdef DWT2_CHECKED
constexpr bool CHECKED_BUILD = true;
#else
constexpr bool CHECKED_BUILD = false;
#endif

__device__ __forceinline__ bool dev_in(unsigned* status, bool in_range) {
    if constexpr (CHECKED_BUILD) {
        if (!in_range && status) atomicOr(status, DEV_CHECK);
        return in_range;
    } else {
        return true;
    }
}

// n elements from ptr lie inside the rows x cols rectangle at base (pitch in
// elements): the pointer arithmetic itself is checked, not only the indices
template <class T>
__device__ __forceinline__ bool dev_in_rect(unsigned* status, const T* ptr, const T* base, int64_t pitch, int64_t rows,
                                            int64_t cols, int n) {
    if constexpr (CHECKED_BUILD) {
        const int64_t off = ptr - base;
        const bool ok = pitch > 0 && off >= 0 && off / pitch < rows && off % pitch + n <= cols;
        return dev_in(status, ok);
    } else {
        return true;
    }
}

// n elements from ptr lie inside the len elements at base
template <class T>
__device__ __forceinline__ bool dev_in_span(unsigned* status, const T* ptr, const T* base, int64_t len, int n) {
    if constexpr (CHECKED_BUILD) {
        const int64_t off = ptr - base;
        return dev_in(status, off >= 0 && off + n <= len);
    } else {
        return true;
    }
}

// a check of this kernel (or of another one sharing the status word) failed
__device__ __forceinline__ bool dev_check_tripped(const unsigned* status) {
    if constexpr (CHECKED_BUILD) {
        return status && (*reinterpret_cast<const volatile unsigned*>(status) & DEV_CHECK) != 0;
    } else {
        return false;
    }
}

// 2-D tiled TMA load of one box into shared memory, completing on `bar`.
// The x coordinate must be a multiple of 4 elements (16 bytes).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Programmatic dependent launch: wait until the grids this one depends on
// have completed and their writes are visible (returns at once when the
// launch had no programmatic dependency), and let the next grid in the stream
// start launching.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" :::); }

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* tm) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}

// ---------------------------------------------------------- conversions
template <class T>
struct Cvt;
template <>
struct Cvt<float> {
    static __device__ __forceinline__ float to(float v) { return v; }
    static __device__ __forceinline__ float from(float v) { return v; }
};
template <>
struct Cvt<int> {
    static __device__ __forceinline__ int to(int v) { return v; }
    static __device__ __forceinline__ int from(int v) { return v; }
};
template <>
struct Cvt<__half> {
    static __device__ __forceinline__ __half to(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ float from(__half v) { return __half2float(v); }
};
template <>
struct Cvt<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 to(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float from(__nv_bfloat16 v) { return __bfloat162float(v); }
};

// two adjacent elements as one vector store (caller guarantees alignment)
template <class T>
__device__ __forceinline__ void st_pair(T* p, T a, T b);
template <>
__device__ __forceinline__ void st_pair<float>(float* p, float a, float b) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
template <>
__device__ __forceinline__ void st_pair<int>(int* p, int a, int b) {
    *reinterpret_cast<int2*>(p) = make_int2(a, b);
}
template <>
__device__ __forceinline__ void st_pair<__half>(__half* p, __half a, __half b) {
    *reinterpret_cast<__half2*>(p) = __halves2half2(a, b);
}
template <>
__device__ __forceinline__ void st_pair<__nv_bfloat16>(__nv_bfloat16* p, __nv_bfloat16 a, __nv_bfloat16 b) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __halves2bfloat162(a, b);
}

// Store the lane's two values of one band row: element j0 and j0+1 of the
// row at `rowp`.  ok0 / ok1 say which are inside the band; vec says the pair
// address is aligned for one vector store.
template <class T, class CT>
__device__ __forceinline__ void store_pair(T* rowp, int j0, CT v0, CT v1, bool ok0, bool ok1, bool vec) {
    const T a = Cvt<T>::to(v0), b = Cvt<T>::to(v1);
    if (ok0 && ok1 && vec) {
        st_pair<T>(rowp + j0, a, b);
    } else {
        if (ok0) rowp[j0] = a;
        if (ok1) rowp[j0 + 1] = b;
    }
}

}  // namespace dwt2
