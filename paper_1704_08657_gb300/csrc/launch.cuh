// launch.cuh -- kernel instantiation and launch helpers; included by one
// translation unit per coefficient type.
#pragma once

#include <type_traits>

#include "fused.cuh"
#include "kernels.cuh"

namespace dwt2 {

template <class Pipe, class OutT, int QL, int QR, int NST, int NW, bool SPEC>
int launch_fwd_one(const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p, int grid, cudaStream_t s) {
    auto k = fwd_tma_kernel<Pipe, OutT, QL, QR, NST, NW, SPEC>;
    constexpr size_t smem = fwd_smem_bytes<QL, QR, NST, NW>();
    if (smem > 48 * 1024) {
        static bool done = false;
        if (!done) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            if (e != cudaSuccess) return e;
            done = true;
        }
    }
    if (!p.pdl) {
        k<<<grid, NW * 32, smem, s>>>(box, row, p);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(NW * 32);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, k, box, row, p);
}

// the compiled forward configurations (quads per lane, quad rows per stage,
// stages, warps per block, specialised interior loop); the first is the default
#define DWT2_FWD_CFG_LIST(X) X(0, 2, 3, 3, 4, 0) X(1, 2, 2, 4, 4, 0) X(2, 2, 2, 4, 8, 0) X(3, 2, 2, 4, 8, 1) X(4, 2, 2, 4, 4, 1)

template <class Pipe, class OutT, int QL, int QR, int NST, int NW, bool SPEC>
int launch_group_one(const GroupLaunch& g, int grid, int pdl, cudaStream_t s) {
    auto k = fwd_group_kernel<Pipe, OutT, QL, QR, NST, NW, SPEC>;
    constexpr size_t smem = fwd_smem_bytes<QL, QR, NST, NW>();
    if (smem > 48 * 1024) {
        static bool done = false;
        if (!done) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            if (e != cudaSuccess) return e;
            done = true;
        }
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(NW * 32);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&lc, k, g);
}

template <template <int, int> class PipeT, int S, class OutT>
int launch_group_cfgs(const GroupLaunch& g, int grid, const FwdCfg& c, int pdl, cudaStream_t s) {
#define DWT2_X(I_, QL_, QR_, NST_, NW_, SP_)                                             \
    if (c.ql == QL_ && c.qr == QR_ && c.nst == NST_ && c.nw == NW_ && c.spec == SP_) \
        return launch_group_one<PipeT<S, QL_>, OutT, QL_, QR_, NST_, NW_, SP_ != 0>(g, grid, pdl, s);
    DWT2_FWD_CFG_LIST(DWT2_X)
#undef DWT2_X
    return cudaErrorInvalidValue;
}

template <class OutT>
int launch_group_t(int wav, int scheme, const GroupLaunch& g, int grid, const FwdCfg& c, int pdl, cudaStream_t s) {
    if constexpr (std::is_same<OutT, int>::value) {
        if (wav != WAV_CDF53I) return cudaErrorInvalidValue;
        if (scheme == SCHEME_SEP) return launch_group_cfgs<Fwd53, SCHEME_SEP, int>(g, grid, c, pdl, s);
        if (scheme == SCHEME_NONSEP) return launch_group_cfgs<Fwd53, SCHEME_NONSEP, int>(g, grid, c, pdl, s);
        return cudaErrorInvalidValue;
    } else {
        if (wav == WAV_DD137) {
            if (scheme == SCHEME_NONSEP) return launch_group_cfgs<Fwd137, SCHEME_NONSEP, OutT>(g, grid, c, pdl, s);
            if (scheme == SCHEME_REDUCED) return launch_group_cfgs<Fwd137, SCHEME_REDUCED, OutT>(g, grid, c, pdl, s);
            if (scheme == SCHEME_SEP) return launch_group_cfgs<Fwd137, SCHEME_SEP, OutT>(g, grid, c, pdl, s);
            return cudaErrorInvalidValue;
        }
        if (wav != WAV_CDF97) return cudaErrorInvalidValue;
        if (scheme == SCHEME_NONSEP) return launch_group_cfgs<Fwd97, SCHEME_NONSEP, OutT>(g, grid, c, pdl, s);
        if (scheme == SCHEME_REDUCED) return launch_group_cfgs<Fwd97, SCHEME_REDUCED, OutT>(g, grid, c, pdl, s);
        if (scheme == SCHEME_SEP) return launch_group_cfgs<Fwd97, SCHEME_SEP, OutT>(g, grid, c, pdl, s);
        if (scheme == SCHEME_POLYCONV) return launch_group_cfgs<Fwd97S, SCHEME_POLYCONV, OutT>(g, grid, c, pdl, s);
        if (scheme == SCHEME_CONV) return launch_group_cfgs<Fwd97S, SCHEME_CONV, OutT>(g, grid, c, pdl, s);
        if (scheme == SCHEME_NSCONV) return launch_group_cfgs<Fwd97S, SCHEME_NSCONV, OutT>(g, grid, c, pdl, s);
        return cudaErrorInvalidValue;
    }
}

template <class Pipe, class OutT, int QL, int QR, int NST, int NW, bool SPEC>
int occupancy_fwd_one() {
    int n = 0;
    auto k = fwd_tma_kernel<Pipe, OutT, QL, QR, NST, NW, SPEC>;
    constexpr size_t smem = fwd_smem_bytes<QL, QR, NST, NW>();
    // above 48 KB the kernel must be allowed its shared memory before the
    // occupancy query counts it (the launch sets the same attribute)
    if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NW * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <template <int, int> class PipeT, int S, class OutT>
int occupancy_fwd_cfgs(const FwdCfg& c) {
#define DWT2_X(I_, QL_, QR_, NST_, NW_, SP_)                                             \
    if (c.ql == QL_ && c.qr == QR_ && c.nst == NST_ && c.nw == NW_ && c.spec == SP_) \
        return occupancy_fwd_one<PipeT<S, QL_>, OutT, QL_, QR_, NST_, NW_, SP_ != 0>();
    DWT2_FWD_CFG_LIST(DWT2_X)
#undef DWT2_X
    return 0;
}

template <class OutT>
int occupancy_forward_t(int wav, int scheme, const FwdCfg& c) {
    if constexpr (std::is_same<OutT, int>::value) {
        if (scheme == SCHEME_SEP) return occupancy_fwd_cfgs<Fwd53, SCHEME_SEP, int>(c);
        return occupancy_fwd_cfgs<Fwd53, SCHEME_NONSEP, int>(c);
    } else {
        if (wav == WAV_DD137) {
            if (scheme == SCHEME_SEP) return occupancy_fwd_cfgs<Fwd137, SCHEME_SEP, OutT>(c);
            if (scheme == SCHEME_REDUCED) return occupancy_fwd_cfgs<Fwd137, SCHEME_REDUCED, OutT>(c);
            return occupancy_fwd_cfgs<Fwd137, SCHEME_NONSEP, OutT>(c);
        }
        if (scheme == SCHEME_NONSEP) return occupancy_fwd_cfgs<Fwd97, SCHEME_NONSEP, OutT>(c);
        if (scheme == SCHEME_REDUCED) return occupancy_fwd_cfgs<Fwd97, SCHEME_REDUCED, OutT>(c);
        if (scheme == SCHEME_POLYCONV) return occupancy_fwd_cfgs<Fwd97S, SCHEME_POLYCONV, OutT>(c);
        if (scheme == SCHEME_CONV) return occupancy_fwd_cfgs<Fwd97S, SCHEME_CONV, OutT>(c);
        if (scheme == SCHEME_NSCONV) return occupancy_fwd_cfgs<Fwd97S, SCHEME_NSCONV, OutT>(c);
        return occupancy_fwd_cfgs<Fwd97, SCHEME_SEP, OutT>(c);
    }
}

// resident blocks per SM of the inner-unit kernel (the one that carries a level)
template <class Pipe, class BT, bool ADJ>
int occupancy_inv_one() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, inv_kernel<Pipe, BT, ADJ, INV_QL, INV_NW, UNITS_INNER>,
                                                      INV_NW * 32, inv_smem_bytes<INV_QR, INV_NST, INV_NW>()) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <class BT>
int occupancy_inverse_t(int wav, int scheme) {
    if constexpr (std::is_same<BT, int>::value) {
        if (scheme == SCHEME_SEP) return occupancy_inv_one<Inv53<SCHEME_SEP, INV_QL>, int, false>();
        return occupancy_inv_one<Inv53<SCHEME_NONSEP, INV_QL>, int, false>();
    } else {
        if (wav == WAV_DD137) {
            if (scheme == SCHEME_SEP) return occupancy_inv_one<Inv137<SCHEME_SEP, INV_QL>, BT, false>();
            return occupancy_inv_one<Inv137<SCHEME_NONSEP, INV_QL>, BT, false>();
        }
        if (scheme == SCHEME_NONSEP) return occupancy_inv_one<Inv97<SCHEME_NONSEP, INV_QL>, BT, false>();
        if (scheme == SCHEME_REDUCED) return occupancy_inv_one<Inv97<SCHEME_REDUCED, INV_QL>, BT, false>();
        return occupancy_inv_one<Inv97<SCHEME_SEP, INV_QL>, BT, false>();
    }
}

template <template <int, int> class PipeT, int S, class OutT>
int launch_fwd_cfgs(const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p, int grid,
                    const FwdCfg& c, cudaStream_t s) {
#define DWT2_X(I_, QL_, QR_, NST_, NW_, SP_)                                             \
    if (c.ql == QL_ && c.qr == QR_ && c.nst == NST_ && c.nw == NW_ && c.spec == SP_) \
        return launch_fwd_one<PipeT<S, QL_>, OutT, QL_, QR_, NST_, NW_, SP_ != 0>(box, row, p, grid, s);
    DWT2_FWD_CFG_LIST(DWT2_X)
#undef DWT2_X
    return cudaErrorInvalidValue;
}

template <class OutT>
int launch_forward_t(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p,
                     int grid, const FwdCfg& c, cudaStream_t s) {
    if constexpr (std::is_same<OutT, int>::value) {
        if (wav != WAV_CDF53I) return cudaErrorInvalidValue;
        if (scheme == SCHEME_SEP) return launch_fwd_cfgs<Fwd53, SCHEME_SEP, int>(box, row, p, grid, c, s);
        if (scheme == SCHEME_NONSEP) return launch_fwd_cfgs<Fwd53, SCHEME_NONSEP, int>(box, row, p, grid, c, s);
        return cudaErrorInvalidValue;
    } else {
        if (wav == WAV_DD137) {
            if (scheme == SCHEME_NONSEP)
                return launch_fwd_cfgs<Fwd137, SCHEME_NONSEP, OutT>(box, row, p, grid, c, s);
            if (scheme == SCHEME_REDUCED)
                return launch_fwd_cfgs<Fwd137, SCHEME_REDUCED, OutT>(box, row, p, grid, c, s);
            if (scheme == SCHEME_SEP) return launch_fwd_cfgs<Fwd137, SCHEME_SEP, OutT>(box, row, p, grid, c, s);
            return cudaErrorInvalidValue;
        }
        if (wav != WAV_CDF97) return cudaErrorInvalidValue;
        if (scheme == SCHEME_NONSEP) return launch_fwd_cfgs<Fwd97, SCHEME_NONSEP, OutT>(box, row, p, grid, c, s);
        if (scheme == SCHEME_REDUCED) return launch_fwd_cfgs<Fwd97, SCHEME_REDUCED, OutT>(box, row, p, grid, c, s);
        if (scheme == SCHEME_SEP) return launch_fwd_cfgs<Fwd97, SCHEME_SEP, OutT>(box, row, p, grid, c, s);
        if (scheme == SCHEME_POLYCONV)
            return launch_fwd_cfgs<Fwd97S, SCHEME_POLYCONV, OutT>(box, row, p, grid, c, s);
        if (scheme == SCHEME_CONV) return launch_fwd_cfgs<Fwd97S, SCHEME_CONV, OutT>(box, row, p, grid, c, s);
        if (scheme == SCHEME_NSCONV)
            return launch_fwd_cfgs<Fwd97S, SCHEME_NSCONV, OutT>(box, row, p, grid, c, s);
        return cudaErrorInvalidValue;
    }
}

template <class Pipe, class OutT>
int launch_pml_one(const PmlLaunch& p, int grid, cudaStream_t s) {
    constexpr size_t smem = fwd_smem_bytes<PML_QL, PML_QR, PML_NST, PML_NW>();
    static_assert(smem <= 48 * 1024, "persistent kernel stages fit the default shared-memory limit");
    if (p.use_tma)
        pml_kernel<Pipe, OutT, PML_QL, PML_QR, PML_NST, PML_NW, true><<<grid, PML_NW * 32, smem, s>>>(p);
    else
        pml_kernel<Pipe, OutT, PML_QL, PML_QR, PML_NST, PML_NW, false><<<grid, PML_NW * 32, smem, s>>>(p);
    return cudaGetLastError();
}

template <class Pipe, class OutT>
int occupancy_pml_one() {
    int a = 0, b = 0;
    constexpr size_t smem = fwd_smem_bytes<PML_QL, PML_QR, PML_NST, PML_NW>();
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &a, pml_kernel<Pipe, OutT, PML_QL, PML_QR, PML_NST, PML_NW, true>, PML_NW * 32, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &b, pml_kernel<Pipe, OutT, PML_QL, PML_QR, PML_NST, PML_NW, false>, PML_NW * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return a < b ? a : b;  // the grid must be resident for either loader
}

// occupancy != 0: return resident blocks per SM instead of launching
template <class OutT>
int launch_pml_t(int wav, int scheme, const PmlLaunch* p, int grid, cudaStream_t s, bool occupancy) {
    if constexpr (std::is_same<OutT, int>::value) {
        if (wav != WAV_CDF53I) return occupancy ? 0 : int(cudaErrorInvalidValue);
        if (scheme == SCHEME_SEP)
            return occupancy ? occupancy_pml_one<Fwd53<SCHEME_SEP, PML_QL>, int>()
                             : launch_pml_one<Fwd53<SCHEME_SEP, PML_QL>, int>(*p, grid, s);
        return occupancy ? occupancy_pml_one<Fwd53<SCHEME_NONSEP, PML_QL>, int>()
                         : launch_pml_one<Fwd53<SCHEME_NONSEP, PML_QL>, int>(*p, grid, s);
    } else {
        if (wav != WAV_CDF97) return occupancy ? 0 : int(cudaErrorInvalidValue);
        if (scheme == SCHEME_NONSEP)
            return occupancy ? occupancy_pml_one<Fwd97<SCHEME_NONSEP, PML_QL>, OutT>()
                             : launch_pml_one<Fwd97<SCHEME_NONSEP, PML_QL>, OutT>(*p, grid, s);
        if (scheme == SCHEME_REDUCED)
            return occupancy ? occupancy_pml_one<Fwd97<SCHEME_REDUCED, PML_QL>, OutT>()
                             : launch_pml_one<Fwd97<SCHEME_REDUCED, PML_QL>, OutT>(*p, grid, s);
        return occupancy ? occupancy_pml_one<Fwd97<SCHEME_SEP, PML_QL>, OutT>()
                         : launch_pml_one<Fwd97<SCHEME_SEP, PML_QL>, OutT>(*p, grid, s);
    }
}

// One launch of the inverse or adjoint units of class CLS of a level (one
// image, or a group); pdl: a programmatic dependent of the previous kernel
// (the edge units of a level, which share no data with its inner units).
inline cudaLaunchConfig_t inv_launch_config(int grid, int pdl, cudaStream_t s, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(INV_NW * 32);
    lc.dynamicSmemBytes = inv_smem_bytes<INV_QR, INV_NST, INV_NW>();
    lc.stream = s;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = pdl ? 1 : 0;
    return lc;
}

template <class Pipe, class BT, bool ADJ>
int launch_inv_one(const InvParams& p, int grid, int pdl, int cls, cudaStream_t s) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t lc = inv_launch_config(grid, pdl, s, attr);
    if (cls == UNITS_INNER) return cudaLaunchKernelEx(&lc, inv_kernel<Pipe, BT, ADJ, INV_QL, INV_NW, UNITS_INNER>, p);
    return cudaLaunchKernelEx(&lc, inv_kernel<Pipe, BT, ADJ, INV_QL, INV_NW, UNITS_EDGE>, p);
}

template <class Pipe, class BT, bool ADJ>
int launch_inv_group_one(const InvGroupLaunch& g, int grid, int pdl, int cls, cudaStream_t s) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t lc = inv_launch_config(grid, pdl, s, attr);
    if (cls == UNITS_INNER) return cudaLaunchKernelEx(&lc, inv_group_kernel<Pipe, BT, ADJ, INV_QL, INV_NW, UNITS_INNER>, g);
    return cudaLaunchKernelEx(&lc, inv_group_kernel<Pipe, BT, ADJ, INV_QL, INV_NW, UNITS_EDGE>, g);
}

template <class BT>
int launch_inv_group_t(int wav, int scheme, const InvGroupLaunch& g, int grid, int pdl, int cls, cudaStream_t s) {
    if constexpr (std::is_same<BT, int>::value) {
        if (wav != WAV_CDF53I) return cudaErrorInvalidValue;
        if (scheme == SCHEME_SEP) return launch_inv_group_one<Inv53<SCHEME_SEP, INV_QL>, int, false>(g, grid, pdl, cls, s);
        return launch_inv_group_one<Inv53<SCHEME_NONSEP, INV_QL>, int, false>(g, grid, pdl, cls, s);
    } else {
        if (wav == WAV_DD137) {
            if (scheme == SCHEME_SEP)
                return launch_inv_group_one<Inv137<SCHEME_SEP, INV_QL>, BT, false>(g, grid, pdl, cls, s);
            return launch_inv_group_one<Inv137<SCHEME_NONSEP, INV_QL>, BT, false>(g, grid, pdl, cls, s);
        }
        if (wav != WAV_CDF97) return cudaErrorInvalidValue;
        if (scheme == SCHEME_NONSEP)
            return launch_inv_group_one<Inv97<SCHEME_NONSEP, INV_QL>, BT, false>(g, grid, pdl, cls, s);
        if (scheme == SCHEME_REDUCED)
            return launch_inv_group_one<Inv97<SCHEME_REDUCED, INV_QL>, BT, false>(g, grid, pdl, cls, s);
        return launch_inv_group_one<Inv97<SCHEME_SEP, INV_QL>, BT, false>(g, grid, pdl, cls, s);
    }
}

template <class BT>
int launch_inverse_t(int wav, int scheme, const InvParams& p, int grid, int pdl, int cls, cudaStream_t s) {
    if constexpr (std::is_same<BT, int>::value) {
        if (wav != WAV_CDF53I) return cudaErrorInvalidValue;
        if (scheme == SCHEME_SEP) return launch_inv_one<Inv53<SCHEME_SEP, INV_QL>, int, false>(p, grid, pdl, cls, s);
        if (scheme == SCHEME_NONSEP) return launch_inv_one<Inv53<SCHEME_NONSEP, INV_QL>, int, false>(p, grid, pdl, cls, s);
        return cudaErrorInvalidValue;
    } else {
        if (wav == WAV_DD137) {
            if (scheme == SCHEME_SEP) return launch_inv_one<Inv137<SCHEME_SEP, INV_QL>, BT, false>(p, grid, pdl, cls, s);
            return launch_inv_one<Inv137<SCHEME_NONSEP, INV_QL>, BT, false>(p, grid, pdl, cls, s);
        }
        if (wav != WAV_CDF97) return cudaErrorInvalidValue;
        if (scheme == SCHEME_NONSEP) return launch_inv_one<Inv97<SCHEME_NONSEP, INV_QL>, BT, false>(p, grid, pdl, cls, s);
        if (scheme == SCHEME_REDUCED) return launch_inv_one<Inv97<SCHEME_REDUCED, INV_QL>, BT, false>(p, grid, pdl, cls, s);
        if (scheme == SCHEME_SEP) return launch_inv_one<Inv97<SCHEME_SEP, INV_QL>, BT, false>(p, grid, pdl, cls, s);
        return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------ fused level pairs
template <class Pipe, class OutT>
int fused_prepare() {
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(fused2_kernel<Pipe, OutT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(fused_smem_bytes()));
        if (e != cudaSuccess) return e;
        done = true;
    }
    return cudaSuccess;
}

// occupancy: return resident blocks per SM instead of launching
template <class Pipe, class OutT>
int launch_fused_one(const CUtensorMap* box, const CUtensorMap* row, const FusedParams* p, int grid, cudaStream_t s,
                     bool occupancy) {
    const int e = fused_prepare<Pipe, OutT>();
    if (occupancy) {
        int n = 0;
        if (e != cudaSuccess || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused2_kernel<Pipe, OutT>,
                                                                              FUSED_THREADS, fused_smem_bytes()) !=
                                    cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return n;
    }
    if (e != cudaSuccess) return e;
    fused2_kernel<Pipe, OutT><<<grid, FUSED_THREADS, fused_smem_bytes(), s>>>(*box, *row, *p);
    return cudaGetLastError();
}

template <class OutT>
int launch_fused_t(int wav, int scheme, const CUtensorMap* box, const CUtensorMap* row, const FusedParams* p,
                   int grid, cudaStream_t s, bool occ) {
    const int bad = occ ? 0 : int(cudaErrorInvalidValue);
    if constexpr (std::is_same<OutT, int>::value) {
        if (wav != WAV_CDF53I) return bad;
        if (scheme == SCHEME_SEP) return launch_fused_one<Fwd53<SCHEME_SEP, 2>, int>(box, row, p, grid, s, occ);
        if (scheme == SCHEME_NONSEP) return launch_fused_one<Fwd53<SCHEME_NONSEP, 2>, int>(box, row, p, grid, s, occ);
        return bad;
    } else {
        if (wav != WAV_CDF97) return bad;
        if (scheme == SCHEME_NONSEP) return launch_fused_one<Fwd97<SCHEME_NONSEP, 2>, OutT>(box, row, p, grid, s, occ);
        if (scheme == SCHEME_REDUCED)
            return launch_fused_one<Fwd97<SCHEME_REDUCED, 2>, OutT>(box, row, p, grid, s, occ);
        if (scheme == SCHEME_SEP) return launch_fused_one<Fwd97<SCHEME_SEP, 2>, OutT>(box, row, p, grid, s, occ);
        return bad;
    }
}

}  // namespace dwt2
